// Gauge-equivariant learned preconditioner for the even-odd Schur system: inference, adjoint,
// weight gradients, Adam training and a preconditioned CGNE, all on the GPU.
//
// Not in the paper (the paper solves with plain CG). Network, for an even-site 5D residual r:
//   u = A^{-1} r ;  v_c = A^{-1} sum_d W1[c,d] T_d u  (odd) ;  M r = W0 u + 1/4 A^{-1} sum_{c,d} W2[c,d] T_d v_c
// T_d is parallel transport by one link (d < 4: U_d(x) psi(x+d); d >= 4: U(x-d)^dag psi(x-d)), the
// W are 4x4 complex spin matrices (gauge equivariant). The initial weights make M the two-term
// Neumann series of S^{-1}. The channel mixing of a layer is, for every (site, s, colour) row,
// a product of the row of transported inputs (C_in x 8 directions x 4 spins, complex) with the
// weight block; it runs on the tensor cores as a real GEMM in BF16 with FP32 accumulation
// (mma.sync m16n8k16), K = 64 C_in, N = 8 C_out. A warp owns the 96 rows of its own 32 threads,
// so the rows it writes to shared memory are the rows it multiplies (no CTA barrier needed).
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "field_access.cuh"
#include "tcgen05.cuh"

namespace odwf {

int spb_for(int Ns);
int ensure_workspace(odwf_s* h, int inner);
int solve_core(odwf_s* h, double m1, double m2, const odwf_solve_opts* opts, odwf_solve_stats* stats,
               cudaStream_t st);
bool coef_host(const odwf_s* h, double m1, double m2, std::vector<double>& host, std::string& err);

constexpr int kMaxC = 2;          // hidden channels
constexpr int kXStride = 24;      // bf16 per A-operand row in shared memory (16 used, padded)

// Inference intermediates: the two-channel output of the first layer is stored as BF16 rows, per
// (cb, colour c, s) one 16-byte chunk [re spins 0..3 | im spins 0..3] at ((cb 3 + c) Ns + s), which is
// exactly the A-operand row the second layer feeds to the tensor cores (it rounds its inputs to BF16
// there anyway, so the result is bit-identical to FP32 intermediates at half the bytes).
struct NetLayerArgs {
    unsigned int* fault;     // set to 1 if a bounded wait for the tensor cores ran out (never expected)
    const float* in[kMaxC];  // input channels (FP32 chunk layout, or BF16 rows), opposite parity
    int cin, cout;
    const float* B;          // B operand, FP32 [cin*4 k-tiles][16][8*cout]
    const float* own;        // optional own-parity field for the W0 term
    const float* w0;         // 4x4 complex, [b][a] (re, im), or null
    int own_in_mix;          // 1: out = Mix(c_hop y + W0 own); 0: out = c_hop Mix(y) + W0 own
    float* out[kMaxC];
    const double* mix;       // transposed s-matrices (P_+ then P_-), 2 Ns^2, or null (no mixing)
    float c_hop;
    const float* links;      // FP32 links of the output parity [Vh][8][20]
    const int* nbr;
    int Vh, Ns;
    // the fifth-dimension mixing `mix` in its structured form (sop != SOP_DENSE, Ns = kStructNs)
    int sop;
    SStruct sc;
};

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// out = U psi for the four spins of psi (U: 3 x 3 complex, row-major re/im)
__device__ __forceinline__ void transport_apply(const float u[18], const float psi[24], float out[24]) {
#pragma unroll
    for (int sp = 0; sp < 4; ++sp)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float ur = u[(i * 3 + j) * 2], ui = u[(i * 3 + j) * 2 + 1];
                const float pr = psi[(sp * 3 + j) * 2], pi = psi[(sp * 3 + j) * 2 + 1];
                re = fmaf(ur, pr, fmaf(-ui, pi, re));
                im = fmaf(ur, pi, fmaf(ui, pr, im));
            }
            out[(sp * 3 + i) * 2] = re;
            out[(sp * 3 + i) * 2 + 1] = im;
        }
}

// T_d psi at (cb, s): full 4-spinor parallel transport by the stored link of direction d.
__device__ __forceinline__ void transport4(const float* in, const float* links, const int* nbr, int cb, int s,
                                           int Ns, int d, float out[24]) {
    float psi[24], u[18];
    const int n = __ldg(nbr + (size_t)cb * 8 + d);
    Store<ST_FLOAT>::load(in, nullptr, (size_t)n, s, Ns, psi);
    Links<ST_FLOAT>::load(links, cb, d, u);
    transport_apply(u, psi, out);
}

// The group's links (spb sites x 8 directions x 20 floats), staged once per group by the whole CTA;
// zeros past the last site. The caller synchronises the CTA afterwards.
__device__ __forceinline__ void stage_group_links(const float* links, float* lk, int g, int spb, int Vh, int tid,
                                                  int nth) {
    const float4* src = reinterpret_cast<const float4*>(links);
    float4* dst = reinterpret_cast<float4*>(lk);
    for (int i = tid; i < spb * 8 * 5; i += nth) {
        const int c_ = g * spb + i / 40;
        dst[i] = c_ < Vh ? __ldg(src + (size_t)c_ * 40 + i % 40) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int CIN, int COUT, bool OUTB>
__global__ void __launch_bounds__(256) k_net_layer(NetLayerArgs a) {
    extern __shared__ __align__(16) unsigned char smem_net[];
    const int Ns = a.Ns;
    const int s = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    constexpr int NCOL = 8 * COUT;
    constexpr int KT = CIN * 4;
    // shared memory: [mix 2 Ns^2 floats][X rows * kXStride bf16][Y COUT * rows * 9 floats]; the
    // s-mixing buffer sh (spb Ns 24 floats, 96 bytes per thread) reuses X (144 bytes per thread),
    // which is dead once every warp has passed the barrier that follows its k loop. Y is channel
    // major (rows of 8 + 1 pad floats).
    float* mix = reinterpret_cast<float*>(smem_net);
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(mix + 2 * Ns * Ns);
    const int rows = nth * 3;
    float* Y = reinterpret_cast<float*>(X + (size_t)rows * kXStride);
    float* sh = reinterpret_cast<float*>(X);
    // Ns = 16: warp-local tensor-core s-mixing with its A-fragment table after Y
    const bool tc = Ns == 16;
    uint32_t* afr = reinterpret_cast<uint32_t*>(Y + (size_t)rows * 9 * COUT);
    if (a.mix) {
        for (int i = tid; i < 2 * Ns * Ns; i += nth) mix[i] = (float)a.mix[i];
        if (tc) s_mix16_afrag(a.mix, afr, tid, nth);
    }
    // B fragments for every k-tile and n-tile, kept in registers
    uint32_t bfrag[KT][COUT][2];
#pragma unroll
    for (int kt = 0; kt < KT; ++kt)
#pragma unroll
        for (int nt = 0; nt < COUT; ++nt) {
            const float* Bt = a.B + (size_t)kt * 16 * NCOL;
            const int n = nt * 8 + gid;
            bfrag[kt][nt][0] = pack_bf16(Bt[(2 * tig) * NCOL + n], Bt[(2 * tig + 1) * NCOL + n]);
            bfrag[kt][nt][1] = pack_bf16(Bt[(2 * tig + 8) * NCOL + n], Bt[(2 * tig + 9) * NCOL + n]);
        }
    float w0[32];
    if (a.w0)
#pragma unroll
        for (int k = 0; k < 32; ++k) w0[k] = a.w0[k];
    __syncthreads();

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        __syncthreads();
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        float acc[6][COUT][4];
#pragma unroll
        for (int m = 0; m < 6; ++m)
#pragma unroll
            for (int nt = 0; nt < COUT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[m][nt][q] = 0.f;
#pragma unroll 1
        for (int kt = 0; kt < KT; ++kt) {
            // this thread's 3 rows (colours) of the k-tile: pairs (ci, d) = (2kt + j) / 8, (2kt + j) % 8
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int q = 2 * kt + j, ci = q >> 3, d = q & 7;
                float x[24];
                if (valid) transport4(a.in[ci], a.links, a.nbr, cb, s, Ns, d, x);
                else
#pragma unroll
                    for (int k = 0; k < 24; ++k) x[k] = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // 8 BF16 (re of spins 0..3, then im) = 16 bytes; the row offset (48 bytes per row,
                    // 16 per half) and the X base (8 Ns^2 bytes, Ns even) keep it 16-byte aligned
                    uint4 v;
                    v.x = pack_bf16(x[(0 * 3 + c) * 2], x[(1 * 3 + c) * 2]);
                    v.y = pack_bf16(x[(2 * 3 + c) * 2], x[(3 * 3 + c) * 2]);
                    v.z = pack_bf16(x[(0 * 3 + c) * 2 + 1], x[(1 * 3 + c) * 2 + 1]);
                    v.w = pack_bf16(x[(2 * 3 + c) * 2 + 1], x[(3 * 3 + c) * 2 + 1]);
                    *reinterpret_cast<uint4*>(X + (size_t)(tid * 3 + c) * kXStride + j * 8) = v;
                }
            }
            __syncwarp();
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                const int r0 = warp * 96 + m * 16;
                const uint32_t* x0 = reinterpret_cast<const uint32_t*>(X + (size_t)(r0 + gid) * kXStride);
                const uint32_t* x8 = reinterpret_cast<const uint32_t*>(X + (size_t)(r0 + gid + 8) * kXStride);
                uint32_t af[4] = {x0[tig], x8[tig], x0[tig + 4], x8[tig + 4]};
#pragma unroll
                for (int nt = 0; nt < COUT; ++nt) mma_bf16(acc[m][nt], af, bfrag[kt][nt]);
            }
            __syncwarp();
        }
        // accumulators -> Y rows (warp-private rows)
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int r0 = warp * 96 + m * 16;
#pragma unroll
            for (int nt = 0; nt < COUT; ++nt) {
                float* y0 = Y + (size_t)nt * rows * 9 + (size_t)(r0 + gid) * 9 + 2 * tig;
                float* y8 = Y + (size_t)nt * rows * 9 + (size_t)(r0 + gid + 8) * 9 + 2 * tig;
                y0[0] = acc[m][nt][0];
                y0[1] = acc[m][nt][1];
                y8[0] = acc[m][nt][2];
                y8[1] = acc[m][nt][3];
            }
        }
        __syncwarp();
        float ow[24];
        if (a.own && valid) Store<ST_FLOAT>::load(a.own, nullptr, (size_t)cb, s, Ns, ow);
        else
#pragma unroll
            for (int k = 0; k < 24; ++k) ow[k] = 0.f;
        float wown[24];  // W0 own
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float re = 0.f, im = 0.f;
                if (a.w0) {
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) {
                        const float wr = w0[(b * 4 + aa) * 2], wi = w0[(b * 4 + aa) * 2 + 1];
                        const float xr = ow[(aa * 3 + c) * 2], xi = ow[(aa * 3 + c) * 2 + 1];
                        re = fmaf(wr, xr, fmaf(-wi, xi, re));
                        im = fmaf(wr, xi, fmaf(wi, xr, im));
                    }
                }
                wown[(b * 3 + c) * 2] = re;
                wown[(b * 3 + c) * 2 + 1] = im;
            }
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            float v[24];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float* yr = Y + (size_t)co * rows * 9 + (size_t)(tid * 3 + c) * 9;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    v[(b * 3 + c) * 2] = a.c_hop * yr[b];
                    v[(b * 3 + c) * 2 + 1] = a.c_hop * yr[4 + b];
                }
            }
            if (a.own_in_mix)
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] += wown[k];
            if (a.mix) {
                __syncthreads();
                row24_store(sh + (ls * Ns + s) * 24, v);
                if (tc) {
                    __syncwarp();
                    s_mix16_tc(afr, sh, lane, warp, ls * Ns + s, v, false);
                } else {
                    __syncthreads();
                    s_mix(mix, sh + ls * Ns * 24, s, Ns, v, false);
                }
            }
            if (!a.own_in_mix && co == 0)
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] += wown[k];
            if (valid) {
                if constexpr (OUTB) {
                    uint4* o = reinterpret_cast<uint4*>(a.out[co]) + (size_t)cb * 3 * Ns + s;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uint4 q;
                        q.x = pack_bf16(v[(0 * 3 + c) * 2], v[(1 * 3 + c) * 2]);
                        q.y = pack_bf16(v[(2 * 3 + c) * 2], v[(3 * 3 + c) * 2]);
                        q.z = pack_bf16(v[(0 * 3 + c) * 2 + 1], v[(1 * 3 + c) * 2 + 1]);
                        q.w = pack_bf16(v[(2 * 3 + c) * 2 + 1], v[(3 * 3 + c) * 2 + 1]);
                        o[(size_t)c * Ns] = q;
                    }
                } else {
                    Store<ST_FLOAT>::store(a.out[co], nullptr, (size_t)cb, s, Ns, v);
                }
            }
        }
    }
}

// ---- 1 -> C layer on the fifth-generation tensor cores (tcgen05, Ns = 16) ------------------------
// The same layer as k_net_layer<1, 2, OUTB> for CTAs of 8 sites x 16 slices = 128 threads: the channel
// mixing of every (site, s, colour) row is D = A B with A the row of transported inputs (K = 64: 8
// directions x 4 spins x re/im, BF16) and B the weight block (K x N, N = 16: 2 output channels x 4
// spins x re/im). Per colour the 128 rows of the CTA are one M = 128 tile: the A rows go to shared
// memory in the canonical K-major layout (core matrices of 8 rows x 8 BF16, one K chunk per
// direction; the 8 K chunks of an 8-row group are contiguous, 1024 bytes per group, so the
// descriptor strides are 128 bytes along K and 1024 along M and every K-step of 16 reads inside its
// tile), B likewise (2 groups of 8 columns), converted once per CTA; one thread issues 3 colours x 4
// K-steps of tcgen05.mma
// (K = 16 each) into FP32 accumulators in tensor memory, and after the commit every thread reads its
// own row of D (its own (site, s) outputs of all channels) with tcgen05.ld. No fragment loads and no
// shared-memory staging of the results.
constexpr int kTcRows = 128;                      // M: threads of the CTA
constexpr int kTcK = 64;                          // K of the 1 -> C layer
constexpr int kTcN = 16;                          // N = 8 C_out, C_out = 2
constexpr int kTcABytes = kTcRows * kTcK * 2;     // one colour's A tile (16 KB)
constexpr int kTcBBytes = kTcN * kTcK * 2;        // B (2 KB)
constexpr uint32_t kTcCols = 64;                  // tensor-memory columns: D of 3 colours x 16

__host__ __device__ constexpr size_t layer12_tc_smem() {
    return (size_t)3 * kTcABytes + kTcBBytes + sizeof(uint32_t) * kAfrag16Words + 64;
}

// MINB > 1 asks the compiler for that many resident CTAs of 128 threads per SM (a register cap of
// 65536 / (128 MINB)); MINB = 1 leaves the registers to the compiler.
template <bool OUTB, int MINB>
__global__ void __launch_bounds__(128, MINB) k_net_layer12_tc(NetLayerArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    constexpr int Ns = 16;
    const int s = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5;
    unsigned char* Asm = smem_tc;                                         // 3 colour tiles
    unsigned char* Bsm = smem_tc + 3 * kTcABytes;                         // N x K, K-major
    uint32_t* afr = reinterpret_cast<uint32_t*>(Bsm + kTcBBytes);         // s-mixing fragment table
    uint64_t* bar = reinterpret_cast<uint64_t*>(afr + kAfrag16Words);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    volatile int* ok_s = reinterpret_cast<volatile int*>(tslot + 1);
    float* sh = reinterpret_cast<float*>(Asm);                           // s-mixing rows, after the MMAs

    // B (FP32 [4 k-tiles][16][16], K index kt 16 + kk) -> BF16 [n][k] in core matrices (k/8, n/8)
    for (int i = tid; i < kTcN * kTcK; i += nth) {
        const int n = i % kTcN, k = i / kTcN;
        const float v = __ldg(a.B + (size_t)(k >> 4) * 16 * kTcN + (k & 15) * kTcN + n);
        __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(Bsm + (n >> 3) * 1024 + (k >> 3) * 128 + (n & 7) * 16) + (k & 7);
        *dst = __float2bfloat16_rn(v);
    }
    if (a.mix) s_mix16_afrag(a.mix, afr, tid, nth);
    if (tid == 0) tc_mbar_init(bar, 1);
    if (warp == 0) {
        tmem_alloc(tslot, kTcCols);
        tmem_relinquish();
    }
    float w0[32];
    if (a.w0)
#pragma unroll
        for (int k = 0; k < 32; ++k) w0[k] = a.w0[k];
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    constexpr uint32_t idesc = idesc_bf16_f32(kTcRows, kTcN);
    uint32_t phase = 0;
    bool ok = true;

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        tc_fence_before();
        __syncthreads();  // the previous group's accumulator reads and s-mixing rows are done
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        // A rows: per direction d one 16-byte K chunk (re spins 0..3, im spins 0..3) per colour
#pragma unroll 1
        for (int d = 0; d < 8; ++d) {
            float x[24];
            if (valid) transport4(a.in[0], a.links, a.nbr, cb, s, Ns, d, x);
            else
#pragma unroll
                for (int k = 0; k < 24; ++k) x[k] = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                uint4 v;
                v.x = pack_bf16(x[(0 * 3 + c) * 2], x[(1 * 3 + c) * 2]);
                v.y = pack_bf16(x[(2 * 3 + c) * 2], x[(3 * 3 + c) * 2]);
                v.z = pack_bf16(x[(0 * 3 + c) * 2 + 1], x[(1 * 3 + c) * 2 + 1]);
                v.w = pack_bf16(x[(2 * 3 + c) * 2 + 1], x[(3 * 3 + c) * 2 + 1]);
                *reinterpret_cast<uint4*>(Asm + c * kTcABytes + (tid >> 3) * 1024 + d * 128 + (tid & 7) * 16) = v;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int k = 0; k < kTcK / 16; ++k)
                    umma_bf16(tmem + c * kTcN, smem_desc(Asm + c * kTcABytes + k * 2 * 128, 128, 1024),
                              smem_desc(Bsm + k * 2 * 128, 128, 1024), idesc, k > 0 ? 1u : 0u);
            umma_commit(bar);
        }
        // one thread waits (bounded) and the CTA follows its outcome, so that the warp-collective
        // accumulator loads below run in every warp or in none
        if (tid == 0) {
            const bool done = tc_mbar_wait_bounded(bar, phase);
            if (!done && a.fault) atomicOr(a.fault, 1u);
            *ok_s = done ? 1 : 0;
        }
        __syncthreads();
        if (!*ok_s) {
            ok = false;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        float dv[3][16];
#pragma unroll
        for (int c = 0; c < 3; ++c) tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c * kTcN, dv[c]);

        float ow[24];
        if (a.own && valid) Store<ST_FLOAT>::load(a.own, nullptr, (size_t)cb, s, Ns, ow);
        else
#pragma unroll
            for (int k = 0; k < 24; ++k) ow[k] = 0.f;
        float wown[24];  // W0 own
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float re = 0.f, im = 0.f;
                if (a.w0) {
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) {
                        const float wr = w0[(b * 4 + aa) * 2], wi = w0[(b * 4 + aa) * 2 + 1];
                        const float xr = ow[(aa * 3 + c) * 2], xi = ow[(aa * 3 + c) * 2 + 1];
                        re = fmaf(wr, xr, fmaf(-wi, xi, re));
                        im = fmaf(wr, xi, fmaf(wi, xr, im));
                    }
                }
                wown[(b * 3 + c) * 2] = re;
                wown[(b * 3 + c) * 2 + 1] = im;
            }
#pragma unroll
        for (int co = 0; co < 2; ++co) {
            float v[24];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    v[(b * 3 + c) * 2] = a.c_hop * dv[c][co * 8 + b];
                    v[(b * 3 + c) * 2 + 1] = a.c_hop * dv[c][co * 8 + 4 + b];
                }
            if (a.own_in_mix)
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] += wown[k];
            if (a.mix) {
                __syncwarp();  // the warp's rows of sh are free (previous channel read)
                if (a.sop != SOP_DENSE) {
                    // structured A^{-1} (or its transpose) by the column pass of the site's 16 lanes
                    float* site = sh + ls * kSSite<float>;
                    row24_store(site + s * kSRow<float>, v);
                    __syncwarp();
                    s_struct_col<float, kStructNs>(a.sc, a.sop, site, kSRow<float>, s);
                    __syncwarp();
                    row24_load(site + s * kSRow<float>, v, false);
                } else {
                    row24_store(sh + (size_t)tid * 24, v);
                    __syncwarp();
                    s_mix16_tc(afr, sh, lane, warp, tid, v, false);
                }
            }
            if (!a.own_in_mix && co == 0)
#pragma unroll
                for (int k = 0; k < 24; ++k) v[k] += wown[k];
            if (valid) {
                if constexpr (OUTB) {
                    uint4* o = reinterpret_cast<uint4*>(a.out[co]) + (size_t)cb * 3 * Ns + s;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uint4 q;
                        q.x = pack_bf16(v[(0 * 3 + c) * 2], v[(1 * 3 + c) * 2]);
                        q.y = pack_bf16(v[(2 * 3 + c) * 2], v[(3 * 3 + c) * 2]);
                        q.z = pack_bf16(v[(0 * 3 + c) * 2 + 1], v[(1 * 3 + c) * 2 + 1]);
                        q.w = pack_bf16(v[(2 * 3 + c) * 2 + 1], v[(3 * 3 + c) * 2 + 1]);
                        o[(size_t)c * Ns] = q;
                    }
                } else {
                    Store<ST_FLOAT>::store(a.out[co], nullptr, (size_t)cb, s, Ns, v);
                }
            }
        }
    }
    if (!ok && tid == 0) {
        // the accumulators' MMAs did not report completion within the limit: give them a last bounded
        // wait before the tensor memory is released
        tc_mbar_wait_bounded(bar, phase);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTcCols);
}

// Second layer (2 input channels, 1 output) with the channel mixing BEFORE the transport. Spin
// weights and colour transport act on different indices, so W[c,d] T_d v_c = T_d (W[c,d] v_c) with
// both applied at the neighbour: per direction d the gathered v_0(x+d), v_1(x+d) form one K = 16
// tensor-core step (2 channels x 4 spins x re/im) giving phi_d, which then takes one FP32 transport
// by U_d. That is 8 transports per (site, s) instead of 16. B is direction-major here: k-tile d
// holds W[c,d] for c = 0, 1 (rows c * 8 + spin (re), c * 8 + 4 + spin (im)).
// The transport runs where the mma leaves phi_d: the A rows are ordered colour-major within a warp
// (row 96 warp + 32 colour + lane) and the B columns as (spin, re/im) pairs, so the D fragment of
// lane (gid, tig) in m-tile (colour c, half h) is phi_d(thread 16 h + gid [+ 8], colour c, spin tig)
// as one complex number. Each lane therefore holds all three colours of one spin for four threads
// of its warp, applies U_d to them and keeps the sums in registers across the eight directions; one
// shared-memory transpose per site group (not one per direction) hands every thread its own spinor.
// CTAs of 128 threads, MINB resident per SM asked of the compiler (4: at most 128 registers)
template <bool INB, int MINB>
__global__ void __launch_bounds__(128, MINB) k_net_layer_mt(NetLayerArgs a) {
    extern __shared__ __align__(16) unsigned char smem_net[];
    const int Ns = a.Ns;
    const int s = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    // shared memory: [mix][X rows * kXStride bf16][links of the group's sites, spb x 8 x 20 floats]
    // [s-mixing fragment table]; sh (rows of 24 floats, the transpose and the s-mixing) reuses X
    float* mix = reinterpret_cast<float*>(smem_net);
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(mix + 2 * Ns * Ns);
    const int rows = nth * 3;
    float* sh = reinterpret_cast<float*>(X);
    float* lk = reinterpret_cast<float*>(X + (size_t)rows * kXStride);
    // Ns = 16: warp-local tensor-core s-mixing with its A-fragment table after the links
    const bool tc = Ns == 16;
    uint32_t* afr = reinterpret_cast<uint32_t*>(lk + (size_t)spb * 8 * 20);
    if (a.mix) {
        for (int i = tid; i < 2 * Ns * Ns; i += nth) mix[i] = (float)a.mix[i];
        if (tc) s_mix16_afrag(a.mix, afr, tid, nth);
    }
    // B columns in (spin, re/im) order: fragment column n = 2 spin + re/im is stored column
    // (re/im) 4 + spin
    uint32_t bfrag[8][2];
    const int bcol = (gid & 1) * 4 + (gid >> 1);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const float* Bt = a.B + (size_t)d * 16 * 8;
        bfrag[d][0] = pack_bf16(Bt[(2 * tig) * 8 + bcol], Bt[(2 * tig + 1) * 8 + bcol]);
        bfrag[d][1] = pack_bf16(Bt[(2 * tig + 8) * 8 + bcol], Bt[(2 * tig + 9) * 8 + bcol]);
    }
    __syncthreads();

    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        __syncthreads();
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        // this lane's sums: acc[h][e][colour][re, im] of spin tig for thread 16 h + gid + 8 e
        float acc[2][2][3][2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e)
#pragma unroll
                for (int i = 0; i < 3; ++i) acc[h][e][i][0] = acc[h][e][i][1] = 0.f;
        // the group's links, all eight directions, staged once
        stage_group_links(a.links, lk, g, spb, a.Vh, tid, nth);
        __syncthreads();
        // site (within the group) of each thread this lane serves
        int lsite[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) lsite[h][e] = (warp * 32 + 16 * h + gid + 8 * e) / Ns;
#pragma unroll 1
        for (int d = 0; d < 8; ++d) {
            const int n = valid ? __ldg(a.nbr + (size_t)cb * 8 + d) : 0;
            // A rows of this thread, colour-major: row 96 warp + 32 c + lane holds
            // [v_0 re s0..3 | v_0 im | v_1 re | v_1 im] of colour c as BF16
#pragma unroll
            for (int ci = 0; ci < 2; ++ci) {
                if constexpr (INB) {
                    // BF16 rows of the first layer: copied to the A-operand rows as they are
                    const uint4* ip = reinterpret_cast<const uint4*>(a.in[ci]) + (size_t)n * 3 * Ns + s;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const uint4 q = valid ? __ldg(ip + (size_t)c * Ns) : make_uint4(0u, 0u, 0u, 0u);
                        *reinterpret_cast<uint4*>(X + (size_t)(warp * 96 + c * 32 + lane) * kXStride + ci * 8) = q;
                    }
                } else {
                    float x[24];
                    if (valid) Store<ST_FLOAT>::load(a.in[ci], nullptr, (size_t)n, s, Ns, x);
                    else
#pragma unroll
                        for (int k = 0; k < 24; ++k) x[k] = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        uint4 q;
                        q.x = pack_bf16(x[(0 * 3 + c) * 2], x[(1 * 3 + c) * 2]);
                        q.y = pack_bf16(x[(2 * 3 + c) * 2], x[(3 * 3 + c) * 2]);
                        q.z = pack_bf16(x[(0 * 3 + c) * 2 + 1], x[(1 * 3 + c) * 2 + 1]);
                        q.w = pack_bf16(x[(2 * 3 + c) * 2 + 1], x[(3 * 3 + c) * 2 + 1]);
                        *reinterpret_cast<uint4*>(X + (size_t)(warp * 96 + c * 32 + lane) * kXStride + ci * 8) = q;
                    }
                }
            }
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // phi_d of the 16 threads 16 h .. 16 h + 15, colours 0..2: D fragments in registers
                float ph[3][4];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int r0 = warp * 96 + c * 32 + 16 * h;
                    const uint32_t* x0 = reinterpret_cast<const uint32_t*>(X + (size_t)(r0 + gid) * kXStride);
                    const uint32_t* x8 = reinterpret_cast<const uint32_t*>(X + (size_t)(r0 + gid + 8) * kXStride);
                    uint32_t af[4] = {x0[tig], x8[tig], x0[tig + 4], x8[tig + 4]};
#pragma unroll
                    for (int q = 0; q < 4; ++q) ph[c][q] = 0.f;
                    mma_bf16(ph[c], af, bfrag[d]);
                }
                // U_d of each served thread's site applied to (phi colours 0..2) of spin tig; the two
                // threads a lane serves in half h share their site when Ns >= 16 (one link load)
                float u[20];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (e == 0 || lsite[h][1] != lsite[h][0]) {
                        const float4* lp = reinterpret_cast<const float4*>(lk) + (lsite[h][e] * 8 + d) * 5;
#pragma unroll
                        for (int q = 0; q < 5; ++q) row4_load(reinterpret_cast<const float*>(lp + q), u + 4 * q);
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float re = acc[h][e][i][0], im = acc[h][e][i][1];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            const float ur = u[(i * 3 + j) * 2], ui = u[(i * 3 + j) * 2 + 1];
                            const float pr = ph[j][2 * e], pi = ph[j][2 * e + 1];
                            re = fmaf(ur, pr, fmaf(-ui, pi, re));
                            im = fmaf(ur, pi, fmaf(ui, pr, im));
                        }
                        acc[h][e][i][0] = re;
                        acc[h][e][i][1] = im;
                    }
                }
            }
            __syncwarp();  // X rows are rewritten by the next direction
        }
        // transpose: every lane writes its sums into the served threads' rows of 24 floats, then each
        // thread reads its own spinor. The rows (sh) alias other warps' X rows: CTA barrier first.
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float* row = sh + (size_t)(warp * 32 + 16 * h + gid + 8 * e) * 24;
#pragma unroll
                for (int i = 0; i < 3; ++i)
                    *reinterpret_cast<float2*>(row + (tig * 3 + i) * 2) = make_float2(acc[h][e][i][0], acc[h][e][i][1]);
            }
        __syncwarp();
        float v[24];
        {
            const float* row = sh + (size_t)tid * 24;
#pragma unroll
            for (int q = 0; q < 6; ++q) row4_load(row + 4 * q, v + 4 * q);
        }
        float ow[24];
        if (a.own && valid) Store<ST_FLOAT>::load(a.own, nullptr, (size_t)cb, s, Ns, ow);
        else
#pragma unroll
            for (int k = 0; k < 24; ++k) ow[k] = 0.f;
        float wown[24];  // W0 own
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float re = 0.f, im = 0.f;
                if (a.w0) {
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) {
                        const float wr = __ldg(a.w0 + (b * 4 + aa) * 2), wi = __ldg(a.w0 + (b * 4 + aa) * 2 + 1);
                        const float xr = ow[(aa * 3 + c) * 2], xi = ow[(aa * 3 + c) * 2 + 1];
                        re = fmaf(wr, xr, fmaf(-wi, xi, re));
                        im = fmaf(wr, xi, fmaf(wi, xr, im));
                    }
                }
                wown[(b * 3 + c) * 2] = re;
                wown[(b * 3 + c) * 2 + 1] = im;
            }
#pragma unroll
        for (int k = 0; k < 24; ++k) v[k] = a.c_hop * v[k] + (a.own_in_mix ? wown[k] : 0.f);
        if (a.mix) {
            __syncthreads();
            if (a.sop != SOP_DENSE && Ns == kStructNs) {
                // structured A^{-1} (or its transpose): the site's 16 threads are lanes of one warp
                float* site = sh + ls * kSSite<float>;
                row24_store(site + s * kSRow<float>, v);
                __syncwarp();
                s_struct_col<float, kStructNs>(a.sc, a.sop, site, kSRow<float>, s);
                __syncwarp();
                row24_load(site + s * kSRow<float>, v, false);
            } else {
                row24_store(sh + (ls * Ns + s) * 24, v);
                if (tc) {
                    __syncwarp();
                    s_mix16_tc(afr, sh, lane, warp, ls * Ns + s, v, false);
                } else {
                    __syncthreads();
                    s_mix(mix, sh + ls * Ns * 24, s, Ns, v, false);
                }
            }
        }
        if (!a.own_in_mix)
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] += wown[k];
        if (valid) Store<ST_FLOAT>::store(a.out[0], nullptr, (size_t)cb, s, Ns, v);
    }
}

// Weight gradients G[co][ci][d][b][a] = sum over output-parity sites, s, colour of
// dl_co[b] conj(x_{ci,d}[a]), x_{ci,d} = T_d in_ci (or in_ci itself when `identity`).
// Per-CTA partial sums (float) to partials[blockIdx.x][P], P = cout*cin*D*32.
struct WgradArgs {
    const float* in[kMaxC];
    const float* dl[kMaxC];
    int cin, cout, identity;
    const float* links;
    const int* nbr;
    int Vh, Ns;
    float* partials;
};

template <int CIN, int COUT, int ND>
__global__ void __launch_bounds__(256) k_net_wgrad(WgradArgs a) {
    constexpr int P = COUT * CIN * ND * 32;
    __shared__ float wacc[8][P];  // per warp
    const int Ns = a.Ns;
    const int s = threadIdx.x, ls = threadIdx.y, spb = blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    for (int i = tid; i < 8 * P; i += nth) (&wacc[0][0])[i] = 0.f;
    __syncthreads();
    for (int g = blockIdx.x; g * spb < a.Vh; g += gridDim.x) {
        const int cb = g * spb + ls;
        const bool valid = cb < a.Vh;
        float dl[COUT][24];
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
            if (valid) Store<ST_FLOAT>::load(a.dl[co], nullptr, (size_t)cb, s, Ns, dl[co]);
            else
#pragma unroll
                for (int k = 0; k < 24; ++k) dl[co][k] = 0.f;
        }
#pragma unroll 1
        for (int ci = 0; ci < CIN; ++ci)
#pragma unroll 1
            for (int d = 0; d < ND; ++d) {
                float x[24];
                if (!valid) {
#pragma unroll
                    for (int k = 0; k < 24; ++k) x[k] = 0.f;
                } else if (a.identity) {
                    Store<ST_FLOAT>::load(a.in[ci], nullptr, (size_t)cb, s, Ns, x);
                } else {
                    transport4(a.in[ci], a.links, a.nbr, cb, s, Ns, d, x);
                }
#pragma unroll
                for (int co = 0; co < COUT; ++co) {
                    float gr[16], gi[16];
#pragma unroll
                    for (int b = 0; b < 4; ++b)
#pragma unroll
                        for (int aa = 0; aa < 4; ++aa) {
                            float re = 0.f, im = 0.f;
#pragma unroll
                            for (int c = 0; c < 3; ++c) {
                                const float dr = dl[co][(b * 3 + c) * 2], di = dl[co][(b * 3 + c) * 2 + 1];
                                const float xr = x[(aa * 3 + c) * 2], xi = x[(aa * 3 + c) * 2 + 1];
                                re = fmaf(dr, xr, fmaf(di, xi, re));   // dl * conj(x)
                                im = fmaf(di, xr, fmaf(-dr, xi, im));
                            }
                            gr[b * 4 + aa] = re;
                            gi[b * 4 + aa] = im;
                        }
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        float vr = gr[k], vi = gi[k];
#pragma unroll
                        for (int off = 16; off > 0; off >>= 1) {
                            vr += __shfl_xor_sync(0xffffffffu, vr, off);
                            vi += __shfl_xor_sync(0xffffffffu, vi, off);
                        }
                        if (lane == 0) {
                            const int base = ((co * CIN + ci) * ND + d) * 32 + 2 * k;
                            wacc[warp][base] += vr;
                            wacc[warp][base + 1] += vi;
                        }
                    }
                }
            }
    }
    __syncthreads();
    for (int i = tid; i < P; i += nth) {
        float t = 0.f;
        for (int w = 0; w < nwarps; ++w) t += wacc[w][i];
        a.partials[(size_t)blockIdx.x * P + i] = t;
    }
}

// gsum[i] (+)= sum over blocks of partials[b][i] in block order (FP64)
__global__ void k_sum_partials(const float* partials, int nblk, int P, double* gsum, int accumulate) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += (double)partials[(size_t)b * P + i];
        gsum[i] = accumulate ? gsum[i] + t : t;
    }
}

// Complex 4x4 helpers on the weight vector (complex128 interleaved):
//   W0 at 0 (16 complex), W1[c][d] at 16 + (c*8+d)*16, W2[c][d] at 16 + C*128 + (c*8+d)*16, each [b][a].
// Build the B operands and the W0 terms of the forward and adjoint layers.
//   which 0: layer 1 forward  (cin 1, cout C):  W1[co][d]
//   which 1: layer 2 forward  (cin C, cout 1):  W2[ci][d]
//   which 2: adjoint layer a  (cin 1, cout C):  1/4 W2[co][d^4]^dag
//   which 3: adjoint layer b  (cin C, cout 1):  W1[ci][d^4]^dag
__global__ void k_net_prep(const double* W, int C, float* B0, float* B1, float* B2, float* B3, float* w0f, float* w0adj) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = 4 * C * 8 * 16;  // (which, channel, d, b*4+a)
    for (int i = tid; i < total; i += gridDim.x * blockDim.x) {
        const int ba = i & 15, d = (i >> 4) & 7, c = (i >> 7) % C, which = i / (C * 128);
        const int b = ba >> 2, aa = ba & 3;
        double wr, wi;
        int co, ci, cout;
        float* B;
        if (which == 0 || which == 1) {
            const size_t off = (which == 0 ? 16 : 16 + (size_t)C * 128) + ((size_t)c * 8 + d) * 16 + b * 4 + aa;
            wr = W[2 * off];
            wi = W[2 * off + 1];
            co = which == 0 ? c : 0;
            ci = which == 0 ? 0 : c;
            cout = which == 0 ? C : 1;
            B = which == 0 ? B0 : B1;
        } else {
            // element [b][a] of the conjugate transpose = conj(element [a][b]) of the source
            const size_t src = (which == 2 ? 16 + (size_t)C * 128 : 16) + ((size_t)c * 8 + (d ^ 4)) * 16 + aa * 4 + b;
            wr = W[2 * src];
            wi = -W[2 * src + 1];
            if (which == 2) {
                wr *= 0.25;
                wi *= 0.25;
            }
            co = which == 2 ? c : 0;
            ci = which == 2 ? 0 : c;
            cout = which == 2 ? C : 1;
            B = which == 2 ? B2 : B3;
        }
        // C -> 1 layers with C = 2 use the direction-major layout of k_net_layer_mt (k-tile d, half ci);
        // the others pair two directions of one channel per k-tile
        const bool dir_major = (cout == 1 && C == 2);
        const int q = ci * 8 + d, kt = dir_major ? d : q >> 1, j = dir_major ? ci : q & 1;
        const int ncol = 8 * cout;
        float* Bt = B + (size_t)kt * 16 * ncol;
        Bt[(j * 8 + aa) * ncol + co * 8 + b] = (float)wr;
        Bt[(j * 8 + 4 + aa) * ncol + co * 8 + b] = (float)-wi;
        Bt[(j * 8 + aa) * ncol + co * 8 + 4 + b] = (float)wi;
        Bt[(j * 8 + 4 + aa) * ncol + co * 8 + 4 + b] = (float)wr;
    }
    if (tid < 16) {
        const int b = tid >> 2, aa = tid & 3;
        w0f[2 * tid] = (float)W[2 * tid];
        w0f[2 * tid + 1] = (float)W[2 * tid + 1];
        w0adj[2 * tid] = (float)W[2 * (aa * 4 + b)];
        w0adj[2 * tid + 1] = (float)-W[2 * (aa * 4 + b) + 1];
    }
}

// Adam on the complex weights (treated as 2P reals); g is dL/dconj(W), whose real/imaginary parts
// are half the derivatives along Re W / Im W.
__global__ void k_adam(double* W, const double* g, double* m1, double* m2, int n, double lr, double b1, double b2,
                       double eps, int t) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double gi = 2.0 * g[i];
        m1[i] = b1 * m1[i] + (1 - b1) * gi;
        m2[i] = b2 * m2[i] + (1 - b2) * gi * gi;
        const double mh = m1[i] / (1 - pow(b1, (double)t)), vh = m2[i] / (1 - pow(b2, (double)t));
        W[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

// delta = (out - e) * inv_ne ; partial |out - e|^2 per block (deterministic grid sum via k_sum_partials)
__global__ void k_resid_scale(const float* out, const float* e, float* delta, size_t n, float inv_ne, float* part) {
    __shared__ float ws[32];
    float acc = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float dd = out[i] - e[i];
        delta[i] = dd * inv_ne;
        acc = fmaf(dd, dd, acc);
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        part[blockIdx.x] = t;
    }
}

__global__ void k_scale_f(float* x, size_t n, float c) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] *= c;
}

}  // namespace odwf

// ================================================================================================
// Host side
// ================================================================================================
using namespace odwf;

struct odwf_net_s {
    odwf_s* h = nullptr;
    int C = 2;
    int P = 0;            // complex parameters
    double* W = nullptr;  // device complex128 weights
    double *m1 = nullptr, *m2 = nullptr, *grad = nullptr;
    int adam_t = 0;
    float *B0 = nullptr, *B1 = nullptr, *B2 = nullptr, *B3 = nullptr, *w0f = nullptr, *w0adj = nullptr;
    bool prepped = false;
    double cm1 = -1, cm2 = -1;
    bool use_tc = true;      // the tcgen05 1 -> 2 layer at Ns = 16 (ODWF_TCGEN05=0: the mma.sync layer)
    // register caps of the two layers (ODWF_NET_OCC=<tc>:<mt>): resident CTAs of 128 threads asked of the
    // compiler. The tcgen05 layer at 4 (128 registers, 16 bytes spilled) runs 155 us against 170 us at the
    // 156 registers it takes uncapped (3 CTAs per SM); the 2 -> 1 layer at 5 (96 registers) gains 1 %.
    int minb_tc = 4, minb_mt = 4;
    double* mats = nullptr;  // transposed A^{-1} (2 Ns^2) then A^{-T} (2 Ns^2), FP64
    SCoef sc{};              // structured form of the same (for the s-mixing kernel; sc.dev unused)
    // FP32 half fields: u (even), v[C] (odd), t (even), gy (even), gh[C] (odd), delta (even)
    float* f[8] = {nullptr};
    float* sf[2] = {nullptr, nullptr};  // preconditioned solve: p (even), t (odd)
    float* partials = nullptr;
    int partials_n = 0;
    std::vector<float*> pairs;  // r_i, e_i (even, FP32)
    std::vector<double> pair_ne;  // |e_i|^2
    std::vector<double> pair_nr;  // |r_i|^2
    int loss_mode = 0;            // ODWF_NET_LOSS_ERROR or ODWF_NET_LOSS_RESIDUAL
};

namespace {

// S or S^dag in FP32 on even fields (defined with the preconditioned solver below)
int schur32(odwf_s* h, const SCoef* c, const float* in, float* tmp, float* out, bool dag, cudaStream_t st);

int net_err(odwf_net_s* n, int code, const std::string& msg) { return set_err(n ? n->h : nullptr, code, msg); }

size_t half32(const odwf_s* h) { return (size_t)h->Vh * h->Ns * 24 * sizeof(float); }

int net_alloc(odwf_net_s* n, void** p, size_t bytes) {
    if (*p) return ODWF_OK;
    if (cudaMalloc(p, bytes) != cudaSuccess) return net_err(n, ODWF_ENOMEM, "cudaMalloc (learned preconditioner)");
    return ODWF_OK;
}

int net_set_masses(odwf_net_s* n, double m1, double m2) {
    if (n->cm1 == m1 && n->cm2 == m2) return ODWF_OK;
    std::vector<double> host;
    std::string err;
    if (!coef_host(n->h, m1, m2, host, err)) return net_err(n, ODWF_EINVAL, err);
    const int NN = n->h->Ns * n->h->Ns;
    std::vector<double> m(4 * (size_t)NN);
    // coef_host order: 2 A+^{-1}, 3 A-^{-1}, 6 A+^{-T}, 7 A-^{-T}
    std::memcpy(m.data(), host.data() + 2 * NN, sizeof(double) * 2 * NN);
    std::memcpy(m.data() + 2 * NN, host.data() + 6 * NN, sizeof(double) * 2 * NN);
    int rc = net_alloc(n, (void**)&n->mats, sizeof(double) * 4 * NN);
    if (rc) return rc;
    if (cudaMemcpy(n->mats, m.data(), sizeof(double) * 4 * NN, cudaMemcpyHostToDevice) != cudaSuccess)
        return net_err(n, ODWF_ECUDA, "copy mixing matrices");
    n->sc.has_st = !n->h->dense_s && struct_host(n->h, m1, m2, &n->sc.st);
    n->cm1 = m1;
    n->cm2 = m2;
    return ODWF_OK;
}

int net_prep(odwf_net_s* n, cudaStream_t st) {
    if (n->prepped) return ODWF_OK;
    k_net_prep<<<8, 256, 0, st>>>(n->W, n->C, n->B0, n->B1, n->B2, n->B3, n->w0f, n->w0adj);
    n->prepped = true;
    return cuda_check(n->h, cudaGetLastError(), "k_net_prep");
}

int grid_for_groups(odwf_s* h, int occ) {
    const int spb = spb_for(h->Ns);
    const int groups = (h->Vh + spb - 1) / spb;
    int g = h->num_sms * occ;
    return g > groups ? groups : (g < 1 ? 1 : g);
}

// cout D-fragment row sets, or (cout == 0) the 2 -> 1 layer's layout: no D-fragment rows (its sums
// stay in registers) and the group's staged links instead; then the s-mixing fragment table
size_t layer_smem(const odwf_s* h, int cout) {
    const int spb = spb_for(h->Ns), nth = spb * h->Ns, rows = nth * 3;
    return sizeof(float) * 2 * h->Ns * h->Ns + sizeof(__nv_bfloat16) * (size_t)rows * kXStride +
           sizeof(float) * (size_t)rows * 9 * cout + (cout == 0 ? sizeof(float) * (size_t)spb * 8 * 20 : 0) +
           (h->Ns == 16 ? sizeof(uint32_t) * kAfrag16Words : 0);
}

// one layer; `parity` is the output parity
// `bf16`: inference intermediates (the 1 -> 2 layer writes, the 2 -> 1 layer reads BF16 rows)
int net_layer(odwf_net_s* n, int parity, int cin, int cout, const float* const* in, const float* B, const float* own,
              const float* w0, int own_in_mix, float* const* out, const double* mix, float c_hop, cudaStream_t st,
              int bf16 = 0) {
    odwf_s* h = n->h;
    NetLayerArgs a{};
    for (int i = 0; i < cin; ++i) a.in[i] = in[i];
    for (int i = 0; i < cout; ++i) a.out[i] = out[i];
    a.cin = cin;
    a.cout = cout;
    a.B = B;
    a.own = own;
    a.w0 = w0;
    a.own_in_mix = own_in_mix;
    a.mix = mix;
    a.c_hop = c_hop;
    a.links = h->U32[parity];
    a.nbr = h->nbr[parity];
    a.Vh = h->Vh;
    a.Ns = h->Ns;
    // the structured form of A^{-1} / A^{-T} (n->mats / n->mats + 2 Ns^2) where it exists
    a.sop = SOP_DENSE;
    if (mix && n->sc.has_st && h->Ns == kStructNs) {
        a.sc = n->sc.st;
        a.sop = (mix == n->mats) ? SOP_AINV : (SOP_AINV | SOP_T);
    }
    const int spb = spb_for(h->Ns);
    // the 2 -> 1 layer keeps its transport sums in registers and needs no D-fragment rows (cout 0)
    const size_t smem = layer_smem(h, (cin == 2 && cout == 1) ? 0 : cout);
    const dim3 blk(h->Ns, spb);
    auto launch = [&](void (*fn)(NetLayerArgs), int kind) -> int {
        // every layer kernel has the same type: one attribute flag per kernel, not per type
        static bool set[7] = {false, false, false, false, false, false, false};
        if (!set[kind]) {
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            set[kind] = true;
        }
        int occ = 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, h->Ns * spb, smem);
        const int key = 2000000 + (bf16 ? 1000 : 0) + cin * 100 + cout * 10 + (own ? 1 : 0);
        cudaEvent_t ev0 = nullptr;
        if (h->prof) prof_begin(h, key, st, &ev0);
        fn<<<grid_for_groups(h, occ < 1 ? 1 : occ), blk, smem, st>>>(a);
        if (h->prof) prof_end(h, key, st, ev0);
        return cuda_check(h, cudaGetLastError(), "k_net_layer");
    };
    if (cin == 1 && cout == 2 && h->Ns == 16 && spb == 8 && n->use_tc) {
        // the tcgen05 layer: its own shared-memory layout and a bounded wait (read by check_fault)
        a.fault = h->fault;
        h->staged_used = true;
        const bool cap = n->minb_tc > 1;
        auto fn = bf16 ? (cap ? k_net_layer12_tc<true, 4> : k_net_layer12_tc<true, 1>)
                       : (cap ? k_net_layer12_tc<false, 4> : k_net_layer12_tc<false, 1>);
        const int vi = (bf16 ? 1 : 0) + (cap ? 2 : 0);
        static bool set_tc[4] = {false, false, false, false};
        const size_t smem_tc = layer12_tc_smem();
        if (!set_tc[vi]) {
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tc);
            set_tc[vi] = true;
        }
        // resident CTAs per SM from the kernel's registers, its shared memory and its tensor-memory columns
        static int occ_tcv[4] = {0, 0, 0, 0};
        int& occ_tc = occ_tcv[vi];
        if (occ_tc == 0) {
            cudaFuncAttributes fa{};
            int dev = 0, smem_sm = 0;
            cudaFuncGetAttributes(&fa, fn);
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            const int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * 128) : 1;
            const int by_smem = (int)(smem_sm / (smem_tc + 1024));
            const int by_tmem = 512 / (int)kTcCols;
            occ_tc = std::max(1, std::min(by_regs, std::min(by_smem, by_tmem)));
        }
        const int key = 2000000 + (bf16 ? 1000 : 0) + cin * 100 + cout * 10 + (own ? 1 : 0);
        cudaEvent_t ev0 = nullptr;
        if (h->prof) prof_begin(h, key, st, &ev0);
        fn<<<grid_for_groups(h, occ_tc), blk, smem_tc, st>>>(a);
        if (h->prof) prof_end(h, key, st, ev0);
        return cuda_check(h, cudaGetLastError(), "k_net_layer12_tc");
    }
    if (cin == 1 && cout == 2) return bf16 ? launch(k_net_layer<1, 2, true>, 0) : launch(k_net_layer<1, 2, false>, 1);
    if (cin == 2 && cout == 1) {
        if (n->minb_mt > 4)
            return bf16 ? launch(k_net_layer_mt<true, 5>, 5) : launch(k_net_layer_mt<false, 5>, 6);
        return bf16 ? launch(k_net_layer_mt<true, 4>, 2) : launch(k_net_layer_mt<false, 4>, 3);
    }
    if (cin == 1 && cout == 1) return launch(k_net_layer<1, 1, false>, 4);
    return net_err(n, ODWF_EINVAL, "unsupported layer shape");
}

// s-mixing of an FP32 half field with a transposed matrix pair (uses the library's s-mix kernel)
int net_smix(odwf_net_s* n, const float* in, float* out, const double* mt, cudaStream_t st) {
    const bool transposed = (mt != n->mats);  // n->mats + 2 Ns^2 holds A^{-T}
    return launch_smix(n->h, ST_FLOAT, in, out, mt, 1.0, st, nullptr, nullptr, &n->sc,
                       transposed ? (SOP_AINV | SOP_T) : SOP_AINV);
}

// M r (adjoint = 0) or M^dag r (adjoint = 1) on FP32 even fields; uses f[0] (u), f[1..2] (v / gh)
int net_apply_even(odwf_net_s* n, const float* r, float* outp, int adjoint, cudaStream_t st) {
    odwf_s* h = n->h;
    const int NN = h->Ns * h->Ns;
    const double* Ainv = n->mats;
    const double* AinvT = n->mats + 2 * NN;
    int rc = net_prep(n, st);
    if (rc) return rc;
    float* v[2] = {n->f[1], n->f[2]};
    // two channels: BF16 intermediates between the layers (one channel keeps the FP32 path)
    const int bf = n->C == 2 ? 1 : 0;
    if (!adjoint) {
        if ((rc = net_smix(n, r, n->f[0], Ainv, st))) return rc;
        const float* in1[1] = {n->f[0]};
        if ((rc = net_layer(n, 1, 1, n->C, in1, n->B0, nullptr, nullptr, 0, v, Ainv, 1.f, st, bf))) return rc;
        const float* in2[2] = {v[0], v[1]};
        float* o[1] = {outp};
        return net_layer(n, 0, n->C, 1, in2, n->B1, n->f[0], n->w0f, 0, o, Ainv, 0.25f, st, bf);
    }
    // M^dag g = A^{-T} [ W0^dag g + sum T^dag W1^dag A^{-T} sum T^dag (W2^dag / 4) A^{-T} g ]
    if ((rc = net_smix(n, r, n->f[0], AinvT, st))) return rc;  // gy * 4
    const float* in1[1] = {n->f[0]};
    if ((rc = net_layer(n, 1, 1, n->C, in1, n->B2, nullptr, nullptr, 0, v, AinvT, 1.f, st, bf))) return rc;
    const float* in2[2] = {v[0], v[1]};
    float* o[1] = {outp};
    return net_layer(n, 0, n->C, 1, in2, n->B3, r, n->w0adj, 1, o, AinvT, 1.f, st, bf);
}

int wgrad(odwf_net_s* n, int parity, int cin, int cout, int identity, const float* const* in, const float* const* dl,
          double* gsum, int accumulate, cudaStream_t st) {
    odwf_s* h = n->h;
    WgradArgs a{};
    for (int i = 0; i < cin; ++i) a.in[i] = in[i];
    for (int i = 0; i < cout; ++i) a.dl[i] = dl[i];
    a.cin = cin;
    a.cout = cout;
    a.identity = identity;
    a.links = h->U32[parity];
    a.nbr = h->nbr[parity];
    a.Vh = h->Vh;
    a.Ns = h->Ns;
    a.partials = n->partials;
    const int spb = spb_for(h->Ns);
    const int nd = identity ? 1 : 8;
    const int P = cout * cin * nd * 32;
    int grid = grid_for_groups(h, 2);
    if ((size_t)grid * P > (size_t)n->partials_n) grid = n->partials_n / P;
    const dim3 blk(h->Ns, spb);
    if (identity && cin == 1 && cout == 1) k_net_wgrad<1, 1, 1><<<grid, blk, 0, st>>>(a);
    else if (!identity && cin == 2 && cout == 1) k_net_wgrad<2, 1, 8><<<grid, blk, 0, st>>>(a);
    else if (!identity && cin == 1 && cout == 2) k_net_wgrad<1, 2, 8><<<grid, blk, 0, st>>>(a);
    else return net_err(n, ODWF_EINVAL, "unsupported gradient shape");
    int rc = cuda_check(h, cudaGetLastError(), "k_net_wgrad");
    if (rc) return rc;
    k_sum_partials<<<(P + 255) / 256, 256, 0, st>>>(n->partials, grid, P, gsum, accumulate);
    return cuda_check(h, cudaGetLastError(), "k_sum_partials");
}

// Loss and gradient over the stored pairs; grad (device, complex128 [P]) overwritten.
int net_loss_grad(odwf_net_s* n, double* loss_out, cudaStream_t st) {
    odwf_s* h = n->h;
    const int C = n->C, NN = h->Ns * h->Ns;
    const double* Ainv = n->mats;
    const double* AinvT = n->mats + 2 * NN;
    if (n->loss_mode == ODWF_NET_LOSS_ERROR)
        for (double ne : n->pair_ne)
            if (!(ne > 0.0)) return set_err(h, ODWF_EINVAL, "error loss: the training pairs were set without e");
    int rc = net_prep(n, st);
    if (rc) return rc;
    // gradient layout in doubles: W0 (32), W1 (C*8*32), W2 (C*8*32) -- the wgrad kernels write
    // [co][ci][d][b][a] (re, im), which matches W1[c][d] (co = c) and W2[ci][d] (co = 0) directly
    double* g0 = n->grad;
    double* g1 = n->grad + 32;
    double* g2 = n->grad + 32 + (size_t)C * 8 * 32;
    float *u = n->f[0], *v0 = n->f[1], *v1 = n->f[2], *out = n->f[3], *gy = n->f[4], *gh0 = n->f[5], *gh1 = n->f[6],
          *delta = n->f[7];
    const size_t nreal = (size_t)h->Vh * h->Ns * 24;
    std::vector<double> losses;
    const int rb = 512;
    for (size_t i = 0; i < n->pairs.size() / 2; ++i) {
        const float* r = n->pairs[2 * i];
        const float* e = n->pairs[2 * i + 1];
        const int acc = i > 0;
        // forward with saved intermediates
        if ((rc = net_smix(n, r, u, Ainv, st))) return rc;
        float* v[2] = {v0, v1};
        const float* in1[1] = {u};
        if ((rc = net_layer(n, 1, 1, C, in1, n->B0, nullptr, nullptr, 0, v, Ainv, 1.f, st))) return rc;
        const float* in2[2] = {v0, v1};
        float* o[1] = {out};
        if ((rc = net_layer(n, 0, C, 1, in2, n->B1, u, n->w0f, 0, o, Ainv, 0.25f, st))) return rc;
        double* lsum = n->grad + n->P * 2;  // scratch double after the gradient
        if (n->loss_mode == ODWF_NET_LOSS_RESIDUAL) {
            // w = S M r - r (gy), |w|^2 to lsum; delta = S^dag w / |r|^2 = dL/dconj(M r)
            const SCoef* c = get_coef(h, n->cm1, n->cm2);
            if (!c) return ODWF_EINVAL;
            if ((rc = schur32(h, c, out, gh1, gh0, false, st))) return rc;
            k_resid_scale<<<rb, 256, 0, st>>>(gh0, r, gy, nreal, 1.f, n->partials);
            if ((rc = cuda_check(h, cudaGetLastError(), "k_resid_scale"))) return rc;
            k_sum_partials<<<1, 32, 0, st>>>(n->partials, rb, 1, lsum + i, 0);
            if ((rc = schur32(h, c, gy, gh1, delta, true, st))) return rc;
            k_scale_f<<<rb, 256, 0, st>>>(delta, nreal, (float)(1.0 / n->pair_nr[i]));
            if ((rc = cuda_check(h, cudaGetLastError(), "k_scale_f"))) return rc;
        } else {
            const double ne = n->pair_ne[i];
            k_resid_scale<<<rb, 256, 0, st>>>(out, e, delta, nreal, (float)(1.0 / ne), n->partials);
            if ((rc = cuda_check(h, cudaGetLastError(), "k_resid_scale"))) return rc;
            k_sum_partials<<<1, 32, 0, st>>>(n->partials, rb, 1, lsum + i, 0);
        }
        // G0 = sum delta (x) conj(u)
        const float* gin[1] = {u};
        const float* gdl[1] = {delta};
        if ((rc = wgrad(n, 0, 1, 1, 1, gin, gdl, g0, acc, st))) return rc;
        // gy = 1/4 A^{-T} delta (the 1/4 is applied through the G2 / adjoint weights below)
        if ((rc = net_smix(n, delta, gy, AinvT, st))) return rc;
        // G2[ci][d] = sum gy (x) conj(T_d v_ci) / 4 ; computed unscaled, scaled at the end
        const float* vin[2] = {v0, v1};
        const float* gyd[1] = {gy};
        if ((rc = wgrad(n, 0, C, 1, 0, vin, gyd, g2, acc, st))) return rc;
        // gh_c = A^{-T} sum_d T_d^dag (W2[c,d]^dag / 4) gy
        float* gh[2] = {gh0, gh1};
        if ((rc = net_layer(n, 1, 1, C, gyd, n->B2, nullptr, nullptr, 0, gh, AinvT, 1.f, st))) return rc;
        // G1[c][d] = sum gh_c (x) conj(T_d u)
        const float* ghd[2] = {gh0, gh1};
        if ((rc = wgrad(n, 1, 1, C, 0, gin, ghd, g1, acc, st))) return rc;
    }
    // scale G2 by 1/4 on the host copy at read time: done here with a tiny scale through cuBLAS-free loop
    std::vector<double> gh((size_t)n->P * 2 + n->pairs.size() / 2);
    if ((rc = cuda_check(h, cudaMemcpyAsync(gh.data(), n->grad, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost, st),
                         "grad D2H")))
        return rc;
    if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
    for (size_t k = 32 + (size_t)C * 8 * 32; k < (size_t)n->P * 2; ++k) gh[k] *= 0.25;
    if ((rc = cuda_check(h, cudaMemcpyAsync(n->grad, gh.data(), sizeof(double) * n->P * 2, cudaMemcpyHostToDevice, st),
                         "grad H2D")))
        return rc;
    double L = 0.0;
    for (size_t i = 0; i < n->pairs.size() / 2; ++i)
        L += gh[(size_t)n->P * 2 + i] / (n->loss_mode == ODWF_NET_LOSS_RESIDUAL ? n->pair_nr[i] : n->pair_ne[i]);
    if (loss_out) *loss_out = L;
    return cuda_check(h, cudaStreamSynchronize(st), "sync");
}

}  // namespace

// ---- C ABI ---------------------------------------------------------------------------------------
extern "C" int odwf_net_create(odwf_t* h, int channels, odwf_net_t** out) {
    if (!h || !out) return set_err(h, ODWF_EINVAL, "null argument");
    if (channels != 1 && channels != 2) return set_err(h, ODWF_EINVAL, "channels must be 1 or 2");
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    if (spb_for(h->Ns) * h->Ns > 256 || (spb_for(h->Ns) * h->Ns) % 32)
        return set_err(h, ODWF_EINVAL, "unsupported Ns for the learned preconditioner");
    odwf_net_s* n = new odwf_net_s();
    n->h = h;
    n->C = channels;
    if (const char* e = std::getenv("ODWF_TCGEN05")) n->use_tc = (e[0] == '1');
    if (const char* e = std::getenv("ODWF_NET_OCC")) {
        int a = 1, b = 0;
        if (std::sscanf(e, "%d:%d", &a, &b) == 2) {
            n->minb_tc = a > 1 ? 4 : 1;
            n->minb_mt = b > 4 ? 5 : 4;
        }
    }
    n->P = 16 + 2 * channels * 8 * 16;
    const int C = channels;
    int rc = ODWF_OK;
    rc = rc ? rc : net_alloc(n, (void**)&n->W, sizeof(double) * 2 * n->P);
    rc = rc ? rc : net_alloc(n, (void**)&n->m1, sizeof(double) * 2 * n->P);
    rc = rc ? rc : net_alloc(n, (void**)&n->m2, sizeof(double) * 2 * n->P);
    rc = rc ? rc : net_alloc(n, (void**)&n->grad, sizeof(double) * (2 * n->P + 1024));
    for (int w = 0; w < 4 && !rc; ++w) {
        const int cin = (w == 0 || w == 2) ? 1 : C, cout = (w == 0 || w == 2) ? C : 1;
        float** B = w == 0 ? &n->B0 : w == 1 ? &n->B1 : w == 2 ? &n->B2 : &n->B3;
        rc = net_alloc(n, (void**)B, sizeof(float) * cin * 4 * 16 * 8 * cout);
        if (!rc) rc = cuda_check(h, cudaMemset(*B, 0, sizeof(float) * cin * 4 * 16 * 8 * cout), "memset B");
    }
    rc = rc ? rc : net_alloc(n, (void**)&n->w0f, sizeof(float) * 32);
    rc = rc ? rc : net_alloc(n, (void**)&n->w0adj, sizeof(float) * 32);
    for (int i = 0; i < 8 && !rc; ++i) rc = net_alloc(n, (void**)&n->f[i], half32(h));
    n->partials_n = h->num_sms * 4 * 2 * 8 * 8 * 32;
    rc = rc ? rc : net_alloc(n, (void**)&n->partials, sizeof(float) * n->partials_n);
    if (rc) {
        odwf_net_destroy(n);
        return rc;
    }
    // Neumann-series initial weights
    std::vector<double> W(2 * (size_t)n->P, 0.0);
    auto put = [&](size_t base, int b, int a, double re, double im) {
        W[2 * (base + b * 4 + a)] = re;
        W[2 * (base + b * 4 + a) + 1] = im;
    };
    for (int i = 0; i < 4; ++i) put(0, i, i, 1.0, 0.0);
    // chiral-basis gamma matrices: gamma_mu = [[0, B_mu], [B_mu^dag, 0]]
    const double Bre[4][2][2] = {{{0, 0}, {0, 0}}, {{0, -1}, {1, 0}}, {{0, 0}, {0, 0}}, {{1, 0}, {0, 1}}};
    const double Bim[4][2][2] = {{{0, -1}, {-1, 0}}, {{0, 0}, {0, 0}}, {{-1, 0}, {0, 1}}, {{0, 0}, {0, 0}}};
    for (int layer = 0; layer < 2; ++layer)
        for (int mu = 0; mu < 4; ++mu)
            for (int sign = 0; sign < 2; ++sign) {  // sign 0: 1 - gamma (d = mu), 1: 1 + gamma (d = 4 + mu)
                const int d = sign ? 4 + mu : mu;
                const size_t base = 16 + (size_t)layer * C * 128 + (size_t)(0 * 8 + d) * 16;
                const double sg = sign ? 1.0 : -1.0;
                for (int i = 0; i < 4; ++i) put(base, i, i, 1.0, 0.0);
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) {
                        // upper-right block B: element (i, 2 + j); lower-left block B^dag: (2 + i, j)
                        put(base, i, 2 + j, sg * Bre[mu][i][j], sg * Bim[mu][i][j]);
                        put(base, 2 + i, j, sg * Bre[mu][j][i], -sg * Bim[mu][j][i]);
                    }
            }
    if (cudaMemcpy(n->W, W.data(), sizeof(double) * W.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m1, 0, sizeof(double) * 2 * n->P) != cudaSuccess ||
        cudaMemset(n->m2, 0, sizeof(double) * 2 * n->P) != cudaSuccess) {
        odwf_net_destroy(n);
        return set_err(h, ODWF_ECUDA, "net initialisation");
    }
    *out = n;
    return ODWF_OK;
}

extern "C" int odwf_net_destroy(odwf_net_t* n) {
    if (!n) return ODWF_OK;
    if (n->h && n->h->net == n) n->h->net = nullptr;  // detach from the handle's EOFA solves
    void* ps[] = {n->W, n->m1, n->m2, n->grad, n->B0, n->B1, n->B2, n->B3, n->w0f, n->w0adj, n->mats, n->partials};
    for (void* p : ps) cudaFree(p);
    for (float* p : n->f) cudaFree(p);
    for (float* p : n->sf) cudaFree(p);
    for (float* p : n->pairs) cudaFree(p);
    delete n;
    return ODWF_OK;
}

extern "C" int odwf_net_weights(odwf_net_t* n, double* host, int set) {
    if (!n || !host) return ODWF_EINVAL;
    const size_t bytes = sizeof(double) * 2 * n->P;
    cudaError_t e = set ? cudaMemcpy(n->W, host, bytes, cudaMemcpyHostToDevice)
                        : cudaMemcpy(host, n->W, bytes, cudaMemcpyDeviceToHost);
    if (set) {
        n->prepped = false;
        n->adam_t = 0;
        cudaMemset(n->m1, 0, bytes);
        cudaMemset(n->m2, 0, bytes);
    }
    return cuda_check(n->h, e, "net weights copy");
}

extern "C" int odwf_net_num_params(const odwf_net_t* n) { return n ? n->P : 0; }

// M r or M^dag r for a 5D field given in the ABI layout (only even sites are read; odd sites of
// the output are zero). FP32 arithmetic with BF16 tensor-core channel mixing.
extern "C" int odwf_net_apply(odwf_net_t* n, double m1, double m2, const void* r, void* out, int adjoint, void* stream) {
    if (!n || !r || !out) return ODWF_EINVAL;
    odwf_s* h = n->h;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_workspace(h, ST_DOUBLE);
    if (rc) return rc;
    if ((rc = net_set_masses(n, m1, m2))) return rc;
    // pack: even part of r -> FP32 (ws.b_e used as FP32 storage), odd part discarded
    if ((rc = launch_pack5(h, (const double*)r, h->ws.b_e, h->ws.b_o, ST_FLOAT, 0, st))) return rc;
    if ((rc = net_apply_even(n, (const float*)h->ws.b_e, (float*)h->ws.x_e, adjoint, st))) return rc;
    if ((rc = cuda_check(h, cudaMemsetAsync(h->ws.x_o, 0, half32(h), st), "memset"))) return rc;
    return launch_unpack5(h, h->ws.x_e, h->ws.x_o, (double*)out, ST_FLOAT, 0, st);
}

// Training pairs: r_i (ABI 5D fields, even sites used) and, when e == NULL, e_i = S^{-1} r_i from
// the library's own solver (FP32 inner CGNE with FP64 reliable updates, tolerance tol); otherwise
// the given e_i. Replaces earlier pairs.
static void clear_pairs(odwf_net_s* n) {
    for (float* p : n->pairs) cudaFree(p);
    n->pairs.clear();
    n->pair_ne.clear();
    n->pair_nr.clear();
}

static int set_pairs_impl(odwf_net_t* n, double m1, double m2, int npairs, const void* const* r,
                          const void* const* e, double tol, void* stream) {
    odwf_s* h = n->h;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_workspace(h, ST_DOUBLE);
    if (rc) return rc;
    if ((rc = net_set_masses(n, m1, m2))) return rc;
    clear_pairs(n);
    odwf_solve_opts so{tol, 100000, ODWF_PREC_SINGLE, 0.01, 0.0};
    for (int i = 0; i < npairs; ++i) {
        float *rf = nullptr, *ef = nullptr;
        if ((rc = net_alloc(n, (void**)&rf, half32(h))) || (rc = net_alloc(n, (void**)&ef, half32(h)))) return rc;
        n->pairs.push_back(rf);
        n->pairs.push_back(ef);
        if ((rc = launch_pack5(h, (const double*)r[i], rf, h->ws.b_o, ST_FLOAT, 0, st))) return rc;
        if (e && e[i]) {
            if ((rc = launch_pack5(h, (const double*)e[i], ef, h->ws.b_o, ST_FLOAT, 0, st))) return rc;
        } else if (n->loss_mode == ODWF_NET_LOSS_RESIDUAL) {
            // the residual loss never reads e_i: no solve (|e_i|^2 = 0 marks the pair as without e)
            if ((rc = cuda_check(h, cudaMemsetAsync(ef, 0, half32(h), st), "memset"))) return rc;
        } else {
            // D_T x = (r_e, 0) gives x_e = S^{-1} r_e (b_hat = r_e when the odd source vanishes)
            if ((rc = launch_pack5(h, (const double*)r[i], h->ws.b_e, h->ws.b_o, ST_DOUBLE, 0, st))) return rc;
            if ((rc = cuda_check(h, cudaMemsetAsync(h->ws.b_o, 0, half_elems_bytes(h, ST_DOUBLE), st), "memset")))
                return rc;
            const int src = solve_core(h, m1, m2, &so, nullptr, st);
            if (src != ODWF_OK) return src;
            if ((rc = launch_convert(h, h->ws.x_e, ST_DOUBLE, nullptr, ef, ST_FLOAT, nullptr, st))) return rc;
        }
        if ((rc = launch_norm2(h, ef, ST_FLOAT, nullptr, 0, st))) return rc;
        if ((rc = launch_norm2(h, rf, ST_FLOAT, nullptr, 1, st))) return rc;
        CGState hs;
        if ((rc = cuda_check(h, cudaMemcpyAsync(&hs, h->state, sizeof(CGState), cudaMemcpyDeviceToHost, st), "D2H")))
            return rc;
        if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
        if (!(hs.result[1] > 0.0) || !std::isfinite(hs.result[1]))
            return set_err(h, ODWF_EINVAL, "a training vector r_i is zero or not finite on the even sites");
        n->pair_ne.push_back(hs.result[0]);
        n->pair_nr.push_back(hs.result[1]);
    }
    return ODWF_OK;
}

extern "C" int odwf_net_set_pairs(odwf_net_t* n, double m1, double m2, int npairs, const void* const* r,
                                  const void* const* e, double tol, void* stream) {
    if (!n || npairs < 1 || !r) return ODWF_EINVAL;
    const int rc = set_pairs_impl(n, m1, m2, npairs, r, e, tol, stream);
    // on any error no partial pair set stays behind (the loss indexes the pairs' norms by pair)
    if (rc != ODWF_OK) clear_pairs(n);
    return rc;
}

extern "C" int odwf_net_set_loss(odwf_net_t* n, int mode) {
    if (!n || (mode != ODWF_NET_LOSS_ERROR && mode != ODWF_NET_LOSS_RESIDUAL)) return ODWF_EINVAL;
    n->loss_mode = mode;
    return ODWF_OK;
}

// Loss L = sum_i |M r_i - e_i|^2 / |e_i|^2 over the stored pairs and its gradient dL/dconj(W)
// (host, complex128 [P], same layout as the weights; may be NULL).
extern "C" int odwf_net_loss_grad(odwf_net_t* n, double* loss, double* grad_host, void* stream) {
    if (!n || n->pairs.empty()) return ODWF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = net_loss_grad(n, loss, st);
    if (rc) return rc;
    if (grad_host)
        return cuda_check(n->h, cudaMemcpy(grad_host, n->grad, sizeof(double) * 2 * n->P, cudaMemcpyDeviceToHost),
                          "grad D2H");
    return ODWF_OK;
}

// `steps` Adam steps (learning rate lr) on the stored pairs; losses[steps + 1] (may be NULL)
// receives the loss before each step and after the last.
extern "C" int odwf_net_train(odwf_net_t* n, int steps, double lr, double* losses, void* stream) {
    if (!n || n->pairs.empty() || steps < 0) return ODWF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    for (int k = 0; k < steps; ++k) {
        double L = 0.0;
        int rc = net_loss_grad(n, &L, st);
        if (rc) return rc;
        if (losses) losses[k] = L;
        n->adam_t += 1;
        k_adam<<<4, 256, 0, st>>>(n->W, n->grad, n->m1, n->m2, 2 * n->P, lr, 0.9, 0.999, 1e-12, n->adam_t);
        if ((rc = cuda_check(n->h, cudaGetLastError(), "k_adam"))) return rc;
        n->prepped = false;
    }
    if (losses) {
        double L = 0.0;
        int rc = net_loss_grad(n, &L, st);
        if (rc) return rc;
        losses[steps] = L;
    }
    return ODWF_OK;
}

// ---- preconditioned CGNE: S M y = b_hat, accumulating x = M y directly ---------------------------
namespace {

const double* coef_mat(const SCoef* c, int k, int Ns) { return c->dev + (size_t)k * Ns * Ns; }

// FP64: out = bh - S x (even), result[slot] = |out|^2 ; tmp: odd scratch
int residual64(odwf_s* h, const SCoef* c, const void* bh, const void* x, void* tmp, void* out, int slot, cudaStream_t st) {
    HopArgs a{};
    a.in = x;
    a.out = tmp;
    a.mhop = coef_mat(c, 2, h->Ns);
    set_sop(a, c, SOP_AINV);
    a.c_hop = 1.0;
    int rc = launch_hop(h, ST_DOUBLE, 1, true, false, false, EPI_STORE, a, st);
    if (rc) return rc;
    HopArgs b{};
    b.in = tmp;
    b.own = x;
    b.out = out;
    b.mown = coef_mat(c, 0, h->Ns);
    set_sop(b, c, SOP_A);
    b.c_hop = -0.25;
    b.x = const_cast<void*>(bh);
    b.slot = slot;
    return launch_hop(h, ST_DOUBLE, 0, false, true, true, EPI_RESID, b, st);
}

int read_state(odwf_s* h, cudaStream_t st) {
    int rc = cuda_check(h, cudaMemcpyAsync(h->state_host, h->state, sizeof(CGState), cudaMemcpyDeviceToHost, st), "D2H");
    return rc ? rc : cuda_check(h, cudaStreamSynchronize(st), "sync");
}

int write_state(odwf_s* h, cudaStream_t st) {
    int rc = cuda_check(h, cudaMemcpyAsync(h->state, h->state_host, sizeof(CGState), cudaMemcpyHostToDevice, st), "H2D");
    return rc ? rc : cuda_check(h, cudaStreamSynchronize(st), "sync");
}

// b' = R5 g5 b (ABI field b), |b'|^2, b_hat = b'_e + 1/2 H_eo A^{-1} b'_o; x_e = 0, r64 = b_hat and
// |r64|^2. All FP64, in the handle's workspace.
int schur_start(odwf_s* h, const SCoef* c, const void* b, double* bnorm2, double* rr64, cudaStream_t st) {
    Workspace& w = h->ws;
    const size_t b64 = half_elems_bytes(h, ST_DOUBLE);
    int rc;
    // b == nullptr: b' is already packed into ws.b_e / ws.b_o (the EOFA terms' right-hand sides)
    if (b && (rc = launch_pack5(h, (const double*)b, w.b_e, w.b_o, ST_DOUBLE, 1, st))) return rc;
    if ((rc = launch_norm2(h, w.b_e, ST_DOUBLE, nullptr, 0, st))) return rc;
    if ((rc = launch_norm2(h, w.b_o, ST_DOUBLE, nullptr, 1, st))) return rc;
    if ((rc = launch_smix(h, ST_DOUBLE, w.b_o, w.t64, coef_mat(c, 2, h->Ns), 1.0, st, nullptr, nullptr, c, SOP_AINV)))
        return rc;
    {
        HopArgs a{};
        a.in = w.t64;
        a.own = w.b_e;
        a.out = w.bh;
        a.a_own = 1.0;
        a.c_hop = 0.5;
        if ((rc = launch_hop(h, ST_DOUBLE, 0, false, true, false, EPI_STORE, a, st))) return rc;
    }
    if ((rc = read_state(h, st))) return rc;
    *bnorm2 = h->state_host->result[0] + h->state_host->result[1];
    if ((rc = cuda_check(h, cudaMemsetAsync(w.x_e, 0, b64, st), "memset"))) return rc;
    if ((rc = cuda_check(h, cudaMemcpyAsync(w.r64, w.bh, b64, cudaMemcpyDeviceToDevice, st), "copy"))) return rc;
    if ((rc = launch_norm2(h, w.r64, ST_DOUBLE, nullptr, 3, st))) return rc;
    if ((rc = read_state(h, st))) return rc;
    *rr64 = h->state_host->result[3];
    return ODWF_OK;
}

// x_o = A^{-1}(b'_o + 1/2 H_oe x_e), the FP64 true residual |b' - D x|/|b'| of both parities, and
// the unpacked solution x (ABI layout).
int schur_finish(odwf_s* h, const SCoef* c, void* x, double bnorm2, double* res, cudaStream_t st) {
    Workspace& w = h->ws;
    int rc;
    HopArgs a{};
    a.in = w.x_e;
    a.own = w.b_o;
    a.out = w.x_o;
    a.a_own = 1.0;
    a.c_hop = 0.5;
    a.mhop = coef_mat(c, 2, h->Ns);
    set_sop(a, c, SOP_AINV);
    if ((rc = launch_hop(h, ST_DOUBLE, 1, true, true, false, EPI_STORE, a, st))) return rc;
    HopArgs r2{};
    r2.mown = coef_mat(c, 0, h->Ns);
    set_sop(r2, c, SOP_A);
    r2.c_hop = -0.5;
    r2.in = w.x_o;
    r2.own = w.x_e;
    r2.x = w.b_e;
    r2.out = w.r64;
    r2.slot = 0;
    if ((rc = launch_hop(h, ST_DOUBLE, 0, false, true, true, EPI_RESID, r2, st))) return rc;
    r2.in = w.x_e;
    r2.own = w.x_o;
    r2.x = w.b_o;
    r2.out = w.t64;
    r2.slot = 1;
    if ((rc = launch_hop(h, ST_DOUBLE, 1, false, true, true, EPI_RESID, r2, st))) return rc;
    // x == nullptr: the solution stays in ws.x_e / ws.x_o
    if (x && (rc = launch_unpack5(h, w.x_e, w.x_o, (double*)x, ST_DOUBLE, 0, st))) return rc;
    if ((rc = read_state(h, st))) return rc;
    // b = 0: x = 0 solves the system exactly (the iteration never started)
    *res = bnorm2 > 0.0 ? std::sqrt((h->state_host->result[0] + h->state_host->result[1]) / bnorm2) : 0.0;
    return ODWF_OK;
}

// S in FP32 on even fields: out = A in - 1/4 H_eo A^{-1} H_oe in (tmp: odd scratch); dag: S^dag
int schur32(odwf_s* h, const SCoef* c, const float* in, float* tmp, float* out, bool dag, cudaStream_t st) {
    HopArgs a{};
    a.in = in;
    a.out = tmp;
    a.mhop = coef_mat(c, dag ? 6 : 2, h->Ns);
    set_sop(a, c, dag ? (SOP_AINV | SOP_T) : SOP_AINV);
    a.c_hop = 1.0;
    a.g5 = dag ? G5_HOP_IN : 0;
    int rc = launch_hop(h, ST_FLOAT, 1, true, false, false, EPI_STORE, a, st);
    if (rc) return rc;
    HopArgs b2{};
    b2.in = tmp;
    b2.own = in;
    b2.out = out;
    b2.mown = coef_mat(c, dag ? 4 : 0, h->Ns);
    set_sop(b2, c, dag ? (SOP_A | SOP_T) : SOP_A);
    b2.c_hop = -0.25;
    b2.g5 = dag ? (G5_OWN_IN | G5_OUT) : 0;
    return launch_hop(h, ST_FLOAT, 0, false, true, true, EPI_STORE, b2, st);
}

}  // namespace

namespace odwf {
// The network-preconditioned CGNE of eofa_solve_learned with b (ABI field) and x (ABI field) optional:
// b == nullptr takes b' = R5 g5 b already packed into ws.b_e / ws.b_o, x == nullptr leaves the solution
// in ws.x_e / ws.x_o (the layout every EOFA term call reads).
int learned_solve(odwf_s* h, odwf_net_s* n, double m1, double m2, const void* b, void* x,
                  const odwf_solve_opts* opts_in, odwf_solve_stats* stats, cudaStream_t st);
}  // namespace odwf

extern "C" int eofa_solve_learned(odwf_t* h, odwf_net_t* n, double m1, double m2, const void* b, void* x,
                                  const odwf_solve_opts* opts_in, odwf_solve_stats* stats, void* stream) {
    if (!h || !n || !b || !x || n->h != h) return set_err(h, ODWF_EINVAL, "bad argument");
    if (!(m1 > 0.0 && m1 <= 1.0) || !(m2 > 0.0 && m2 <= 1.0)) return set_err(h, ODWF_EINVAL, "masses must lie in (0, 1]");
    return odwf::learned_solve(h, n, m1, m2, b, x, opts_in, stats, (cudaStream_t)stream);
}

extern "C" int odwf_set_preconditioner(odwf_t* h, odwf_net_t* n) {
    if (!h || (n && n->h != h)) return set_err(h, ODWF_EINVAL, "the network belongs to another handle");
    h->net = n;
    return ODWF_OK;
}

int odwf::learned_solve(odwf_s* h, odwf_net_s* n, double m1, double m2, const void* b, void* x,
                        const odwf_solve_opts* opts_in, odwf_solve_stats* stats, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    odwf_solve_opts o{1e-10, 100000, ODWF_PREC_SINGLE, 1e-3, 0.0};
    if (opts_in) o = *opts_in;
    int rc = ensure_workspace(h, ST_DOUBLE);
    if (rc) return rc;
    if ((rc = net_set_masses(n, m1, m2))) return rc;
    for (int i = 0; i < 2 && !rc; ++i) rc = net_alloc(n, (void**)&n->sf[i], half32(h));
    if (rc) return rc;
    const SCoef* c = get_coef(h, m1, m2);
    if (!c) return ODWF_EINVAL;
    Workspace& w = h->ws;
    const size_t b64 = half_elems_bytes(h, ST_DOUBLE), b32 = half32(h);
    float *z = n->f[3], *wv = n->f[4], *mv = n->f[5], *xi = n->f[6], *rho = n->f[7], *p = n->sf[0], *t = n->sf[1];
    double bnorm2 = 0.0, rr64 = 0.0;
    if ((rc = schur_start(h, c, b, &bnorm2, &rr64, st))) return rc;
    if (!std::isfinite(bnorm2) || !std::isfinite(rr64))
        return set_err(h, ODWF_EBREAKDOWN, "non-finite right-hand side (|b|^2 is not finite)");
    const double tol2 = o.tol * o.tol * bnorm2;
    int iters = 0, cycles = 0;
    const double delta = (o.delta > 0 && o.delta < 1) ? o.delta : 1e-3;
    // reliable updates: after the first cycle the search direction and the last beta carry over, so the
    // FP64 residual replaces the FP32 one without discarding the Krylov space (ODWF_NET_RESTART=1 restarts
    // each cycle from p = 0 instead)
    const char* restart_env = std::getenv("ODWF_NET_RESTART");
    const bool restart = restart_env && restart_env[0] == '1';
    double beta_keep = 0.0;
    auto S32 = [&](const float* in, float* out, bool dag) -> int { return schur32(h, c, in, t, out, dag, st); };
    while (rr64 > tol2 && iters < o.maxiter) {
        // cycle: solve S M y = r64 to relative delta, x_inner = M y accumulated directly
        const bool keep = cycles > 0 && !restart;
        if ((rc = launch_convert(h, w.r64, ST_DOUBLE, nullptr, rho, ST_FLOAT, nullptr, st))) return rc;
        if ((rc = cuda_check(h, cudaMemsetAsync(xi, 0, b32, st), "memset"))) return rc;
        if (!keep && (rc = cuda_check(h, cudaMemsetAsync(p, 0, b32, st), "memset"))) return rc;
        CGState& hs = *h->state_host;
        std::memset(&hs, 0, sizeof(CGState));
        hs.rr = rr64;
        hs.rr_max = rr64;
        hs.tol2 = std::max(0.25 * tol2, delta * delta * rr64);
        hs.maxiter = o.maxiter - iters;
        hs.beta = keep ? beta_keep : 0.0;
        if ((rc = write_state(h, st))) return rc;
        // p = M^dag S^dag rho + beta p (beta = 0 in the first cycle)
        if ((rc = S32(rho, wv, true))) return rc;
        if ((rc = net_apply_even(n, wv, mv, 1, st))) return rc;
        {
            HopArgs a{};
            a.own = mv;
            a.a_own = 1.0;
            a.r = p;
            a.state = h->state;
            if ((rc = launch_hop_own_cgb(h, ST_FLOAT, a, st))) return rc;
        }
        int flag = FLAG_RUN;
        while (flag == FLAG_RUN) {
            for (int k = 0; k < 8; ++k) {
                // z = M p ; S z with the CGNE update x += alpha z, rho -= alpha S z
                if ((rc = net_apply_even(n, p, z, 0, st))) return rc;
                HopArgs a{};
                a.in = z;
                a.out = t;
                a.mhop = coef_mat(c, 2, h->Ns);
                set_sop(a, c, SOP_AINV);
                a.c_hop = 1.0;
                a.state = h->state;
                if ((rc = launch_hop(h, ST_FLOAT, 1, true, false, false, EPI_STORE, a, st))) return rc;
                HopArgs b2{};
                b2.in = t;
                b2.own = z;
                b2.mown = coef_mat(c, 0, h->Ns);
                set_sop(b2, c, SOP_A);
                b2.c_hop = -0.25;
                b2.x = xi;
                b2.r = rho;
                b2.state = h->state;
                if ((rc = launch_hop(h, ST_FLOAT, 0, false, true, true, EPI_CG_A, b2, st))) return rc;
                // p = M^dag S^dag rho + beta p
                if ((rc = S32(rho, wv, true))) return rc;
                if ((rc = net_apply_even(n, wv, mv, 1, st))) return rc;
                HopArgs c2{};
                c2.own = mv;
                c2.a_own = 1.0;
                c2.r = p;
                c2.state = h->state;
                if ((rc = launch_hop_own_cgb(h, ST_FLOAT, c2, st))) return rc;
            }
            if ((rc = read_state(h, st))) return rc;
            flag = h->state_host->flag;
        }
        iters += h->state_host->iter;
        beta_keep = h->state_host->beta;
        ++cycles;
        if (flag == FLAG_BREAKDOWN) return set_err(h, ODWF_EBREAKDOWN, "preconditioned CGNE breakdown");
        if ((rc = launch_axpy_to64(h, 1.0, xi, ST_FLOAT, nullptr, (double*)w.x_e, st))) return rc;
        if ((rc = residual64(h, c, w.bh, w.x_e, w.t64, w.r64, 3, st))) return rc;
        if ((rc = read_state(h, st))) return rc;
        rr64 = h->state_host->result[3];
        if (!std::isfinite(rr64)) return set_err(h, ODWF_EBREAKDOWN, "non-finite residual");
    }
    double res = 0.0;
    if ((rc = schur_finish(h, c, x, bnorm2, &res, st))) return rc;
    if ((rc = check_fault(h, st))) return rc;
    if (stats) {
        stats->iters = iters;
        stats->reliable_updates = cycles;
        stats->true_residual = res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!(res <= o.tol)) return set_err(h, ODWF_ENOCONV, "preconditioned solve did not reach tol");
    return ODWF_OK;
}

// ---- flexible GCR on S, right-preconditioned by the network ---------------------------------------
// Inner FP32 iteration (basis of nvec directions, restarted when full or kept as a sliding window of
// the last nvec - 1), with the residual replaced by the FP64
// true residual b_hat - S x whenever it has dropped by opts->delta (defect correction). Step j:
//   z_j = M r (r itself without a network), w_j = S z_j, then classical Gram-Schmidt of w_j against
//   the orthonormal w_0 .. w_{j-1} (the same combination applied to z_j keeps w_j = S z_j), and
//   e += alpha z_j, r -= alpha w_j with alpha = <w_j, r>. One pass computes all inner products of
//   step j (<w_i, w_j>, |w_j|^2, <w_j, r>, <w_i, r>); |w_j - sum beta_i w_i|^2 follows from the
//   orthonormality of the basis and <w_j - sum beta_i w_i, r> from the <w_i, r>.
namespace odwf {

constexpr int kGcrMax = 16;

struct GcrPtrs {
    const float4* p[kGcrMax];
};

template <int NV>
__device__ __forceinline__ void gcr_block_sum(const float* acc, double* out) {
    __shared__ double red[8][NV];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double v = acc[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[wp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// per-block partial sums, doubles [blk][2 (2 K + 2)]: <V_i, w> (i < K), |w|^2 (imaginary part 0),
// <w, r>, <V_i, r> (i < K)
template <int K>
__global__ void __launch_bounds__(256) k_gcr_dots(GcrPtrs V, const float4* __restrict__ w,
                                                  const float4* __restrict__ r, size_t n4, double* partials) {
    constexpr int NV = 2 * (2 * K + 2);
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x) {
        const float4 a = w[k], b = r[k];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float4 v = V.p[i][k];
            acc[2 * i] += v.x * a.x + v.y * a.y + v.z * a.z + v.w * a.w;
            acc[2 * i + 1] += v.x * a.y - v.y * a.x + v.z * a.w - v.w * a.z;
            acc[2 * K + 4 + 2 * i] += v.x * b.x + v.y * b.y + v.z * b.z + v.w * b.w;
            acc[2 * K + 5 + 2 * i] += v.x * b.y - v.y * b.x + v.z * b.w - v.w * b.z;
        }
        acc[2 * K] += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
        acc[2 * K + 2] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
        acc[2 * K + 3] += a.x * b.y - a.y * b.x + a.z * b.w - a.w * b.z;
    }
    gcr_block_sum<NV>(acc, partials + (size_t)blockIdx.x * NV);
}

// out[v] = sum over blocks of partials[b][v]; one warp per value
__global__ void k_gcr_sum(const double* partials, int nblk, int nval, double* out) {
    const int v = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) s += partials[(size_t)b * nval + v];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (threadIdx.x == 0) out[v] = s;
}

__device__ __forceinline__ float4 cmul_sub(float4 a, float br, float bi, float4 v) {
    a.x -= br * v.x - bi * v.y;
    a.y -= br * v.y + bi * v.x;
    a.z -= br * v.z - bi * v.w;
    a.w -= br * v.w + bi * v.z;
    return a;
}

// w_j, z_j <- (w_j - sum beta_i W_i) / n, (z_j - sum beta_i Z_i) / n; r -= alpha w_j; e += alpha z_j
// with alpha = <w_j - sum beta_i W_i, r> / n = (<w_j, r> - sum conj(beta_i) <W_i, r>) / n;
// per-block |r|^2 to rpart. A direction with no component outside the basis is dropped (zeroed).
template <int K>
__global__ void __launch_bounds__(256) k_gcr_update(GcrPtrs W, GcrPtrs Z, const double* __restrict__ sums,
                                                    float4* w, float4* z, float4* r, float4* e, size_t n4,
                                                    double* rpart) {
    const double ww = sums[2 * K];
    double n2 = ww;
    float br[K > 0 ? K : 1], bi[K > 0 ? K : 1];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        br[i] = (float)sums[2 * i];
        bi[i] = (float)sums[2 * i + 1];
        n2 -= sums[2 * i] * sums[2 * i] + sums[2 * i + 1] * sums[2 * i + 1];
    }
    double wr = sums[2 * K + 2], wi = sums[2 * K + 3];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const double b_r = sums[2 * i], b_i = sums[2 * i + 1];
        const double c_r = sums[2 * K + 4 + 2 * i], c_i = sums[2 * K + 5 + 2 * i];
        wr -= b_r * c_r + b_i * c_i;
        wi -= b_r * c_i - b_i * c_r;
    }
    float inv = 0.f, ar = 0.f, ai = 0.f;
    if (ww > 0.0 && n2 > 1e-10 * ww) {
        const double id = 1.0 / sqrt(n2);
        inv = (float)id;
        ar = (float)(wr * id);
        ai = (float)(wi * id);
    }
    float acc[1] = {0.f};
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x) {
        float4 a = w[k], c = z[k];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            a = cmul_sub(a, br[i], bi[i], W.p[i][k]);
            c = cmul_sub(c, br[i], bi[i], Z.p[i][k]);
        }
        a.x *= inv, a.y *= inv, a.z *= inv, a.w *= inv;
        c.x *= inv, c.y *= inv, c.z *= inv, c.w *= inv;
        w[k] = a;
        z[k] = c;
        float4 rr = cmul_sub(r[k], ar, ai, a);
        r[k] = rr;
        acc[0] += rr.x * rr.x + rr.y * rr.y + rr.z * rr.z + rr.w * rr.w;
        const float4 ee = e[k];
        e[k] = make_float4(ee.x + ar * c.x - ai * c.y, ee.y + ar * c.y + ai * c.x, ee.z + ar * c.z - ai * c.w,
                           ee.w + ar * c.w + ai * c.z);
    }
    gcr_block_sum<1>(acc, rpart + blockIdx.x);
}

}  // namespace odwf

namespace {

struct GcrCache {
    int cap = 0;
    float* W[kGcrMax] = {nullptr};
    float* Z[kGcrMax] = {nullptr};
    float *r = nullptr, *e = nullptr, *t = nullptr;
    double *partials = nullptr, *sums = nullptr, *host = nullptr;
    int nblk = 0;
};

void gcr_release(void* p) {
    GcrCache* g = static_cast<GcrCache*>(p);
    if (!g) return;
    for (int i = 0; i < kGcrMax; ++i) {
        cudaFree(g->W[i]);
        cudaFree(g->Z[i]);
    }
    cudaFree(g->r);
    cudaFree(g->e);
    cudaFree(g->t);
    cudaFree(g->partials);
    cudaFree(g->sums);
    if (g->host) cudaFreeHost(g->host);
    delete g;
}

int gcr_ensure(odwf_s* h, int restart, GcrCache** out) {
    if (!h->gcr) {
        GcrCache* g = new GcrCache();
        g->nblk = h->num_sms * 4;
        h->gcr = g;
        h->gcr_free = gcr_release;
        // dots of a step: [nblk][2 (2 K + 2)], K <= kGcrMax - 1: <= 64 nblk; then |r|^2 partials at 64 nblk
        const size_t pb = sizeof(double) * (size_t)g->nblk * 65;
        if (cudaMalloc((void**)&g->r, half32(h)) != cudaSuccess || cudaMalloc((void**)&g->e, half32(h)) != cudaSuccess ||
            cudaMalloc((void**)&g->t, half32(h)) != cudaSuccess || cudaMalloc((void**)&g->partials, pb) != cudaSuccess ||
            cudaMalloc((void**)&g->sums, sizeof(double) * 128) != cudaSuccess ||
            cudaMallocHost((void**)&g->host, sizeof(double) * 8) != cudaSuccess)
            return set_err(h, ODWF_ENOMEM, "GCR work fields");
    }
    GcrCache* g = static_cast<GcrCache*>(h->gcr);
    if (!g->r || !g->e || !g->t || !g->partials || !g->sums || !g->host)
        return set_err(h, ODWF_ENOMEM, "GCR work fields");
    for (; g->cap < restart; ++g->cap)
        if (cudaMalloc((void**)&g->W[g->cap], half32(h)) != cudaSuccess ||
            cudaMalloc((void**)&g->Z[g->cap], half32(h)) != cudaSuccess)
            return set_err(h, ODWF_ENOMEM, "GCR basis");
    *out = g;
    return ODWF_OK;
}

template <int K>
int gcr_step_k(odwf_s* h, GcrCache* g, const int* win, int slot, size_t n4, cudaStream_t st) {
    GcrPtrs PW{}, PZ{};
    for (int i = 0; i < K; ++i) {
        PW.p[i] = reinterpret_cast<const float4*>(g->W[win[i]]);
        PZ.p[i] = reinterpret_cast<const float4*>(g->Z[win[i]]);
    }
    float4* w = reinterpret_cast<float4*>(g->W[slot]);
    float4* z = reinterpret_cast<float4*>(g->Z[slot]);
    cudaEvent_t ev = nullptr;
    if (h->prof) prof_begin(h, 3000100 + K, st, &ev);
    k_gcr_dots<K><<<g->nblk, 256, 0, st>>>(PW, w, reinterpret_cast<const float4*>(g->r), n4, g->partials);
    if (h->prof) prof_end(h, 3000100 + K, st, ev);
    if (h->prof) prof_begin(h, 3000200, st, &ev);
    k_gcr_sum<<<2 * (2 * K + 2), 32, 0, st>>>(g->partials, g->nblk, 2 * (2 * K + 2), g->sums);
    if (h->prof) prof_end(h, 3000200, st, ev);
    if (h->prof) prof_begin(h, 3000300 + K, st, &ev);
    k_gcr_update<K><<<g->nblk, 256, 0, st>>>(PW, PZ, g->sums, w, z, reinterpret_cast<float4*>(g->r),
                                             reinterpret_cast<float4*>(g->e), n4, g->partials + 64 * g->nblk);
    if (h->prof) prof_end(h, 3000300 + K, st, ev);
    return cuda_check(h, cudaGetLastError(), "GCR step");
}

// orthogonalisation of the new direction in basis slot `slot` against the K directions in slots
// win[0 .. K-1] (0 <= K < kGcrMax), and the update of e and r
int gcr_step(odwf_s* h, GcrCache* g, const int* win, int K, int slot, size_t n4, cudaStream_t st) {
    switch (K) {
#define GCR_CASE(KK) \
    case KK: return gcr_step_k<KK>(h, g, win, slot, n4, st);
        GCR_CASE(0) GCR_CASE(1) GCR_CASE(2) GCR_CASE(3) GCR_CASE(4) GCR_CASE(5) GCR_CASE(6) GCR_CASE(7)
        GCR_CASE(8) GCR_CASE(9) GCR_CASE(10) GCR_CASE(11) GCR_CASE(12) GCR_CASE(13) GCR_CASE(14) GCR_CASE(15)
#undef GCR_CASE
    }
    return set_err(h, ODWF_EINVAL, "GCR step out of range");
}

}  // namespace

extern "C" int eofa_solve_gcr(odwf_t* h, odwf_net_t* n, double m1, double m2, const void* b, void* x, int nvec,
                              int truncate, const odwf_solve_opts* opts_in, odwf_solve_stats* stats, void* stream) {
    if (!h || !b || !x || (n && n->h != h)) return set_err(h, ODWF_EINVAL, "bad argument");
    if (!(m1 > 0.0 && m1 <= 1.0) || !(m2 > 0.0 && m2 <= 1.0)) return set_err(h, ODWF_EINVAL, "masses must lie in (0, 1]");
    if (nvec < 1 || nvec > kGcrMax) return set_err(h, ODWF_EINVAL, "nvec must lie in 1..16");
    const int restart = nvec;
    if (!h->have_gauge) return set_err(h, ODWF_EINVAL, "odwf_set_gauge has not been called");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    odwf_solve_opts o{1e-10, 100000, ODWF_PREC_SINGLE, 1e-3, 0.0};
    if (opts_in) o = *opts_in;
    int rc = ensure_workspace(h, ST_DOUBLE);
    if (rc) return rc;
    if (n && (rc = net_set_masses(n, m1, m2))) return rc;
    const SCoef* c = get_coef(h, m1, m2);
    if (!c) return ODWF_EINVAL;
    GcrCache* g = nullptr;
    if ((rc = gcr_ensure(h, restart, &g))) return rc;
    Workspace& w = h->ws;
    const size_t b32 = half32(h), n4 = b32 / sizeof(float4);
    double bnorm2 = 0.0, rr64 = 0.0;
    if ((rc = schur_start(h, c, b, &bnorm2, &rr64, st))) return rc;
    if (!std::isfinite(bnorm2) || !std::isfinite(rr64))
        return set_err(h, ODWF_EBREAKDOWN, "non-finite right-hand side (|b|^2 is not finite)");
    const double tol2 = o.tol * o.tol * bnorm2;
    const double delta = (o.delta > 0 && o.delta < 1) ? o.delta : 1e-3;
    int iters = 0, cycles = 0;
    bool timed_out = false;
    auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    while (rr64 > tol2 && iters < o.maxiter && !timed_out) {
        if ((rc = launch_convert(h, w.r64, ST_DOUBLE, nullptr, g->r, ST_FLOAT, nullptr, st))) return rc;
        if ((rc = cuda_check(h, cudaMemsetAsync(g->e, 0, b32, st), "memset"))) return rc;
        const double target = std::max(0.25 * tol2, delta * delta * rr64);
        double rr = rr64;
        long jt = 0;  // steps of this inner solve
        while (rr > target && iters < o.maxiter && !timed_out) {
            for (int j = 0; j < restart && iters < o.maxiter; ++j, ++iters, ++jt) {
                // restarted: slots 0 .. j-1 then slot j; truncated: the last min(jt, nvec - 1) steps' slots
                int win[kGcrMax], K, slot;
                if (truncate) {
                    slot = (int)(jt % nvec);
                    K = (int)std::min<long>(jt, nvec - 1);
                    for (int i = 0; i < K; ++i) win[i] = (int)((jt - K + i) % nvec);
                } else {
                    slot = j;
                    K = j;
                    for (int i = 0; i < K; ++i) win[i] = i;
                }
                if (n) {
                    if ((rc = net_apply_even(n, g->r, g->Z[slot], 0, st))) return rc;
                } else if ((rc = cuda_check(h, cudaMemcpyAsync(g->Z[slot], g->r, b32, cudaMemcpyDeviceToDevice, st),
                                            "copy"))) {
                    return rc;
                }
                if ((rc = schur32(h, c, g->Z[slot], g->t, g->W[slot], false, st))) return rc;
                if ((rc = gcr_step(h, g, win, K, slot, n4, st))) return rc;
            }
            k_gcr_sum<<<1, 32, 0, st>>>(g->partials + 64 * g->nblk, g->nblk, 1, g->sums + 64);
            if ((rc = cuda_check(h, cudaMemcpyAsync(g->host, g->sums + 64, sizeof(double), cudaMemcpyDeviceToHost, st),
                                 "D2H")))
                return rc;
            if ((rc = cuda_check(h, cudaStreamSynchronize(st), "sync"))) return rc;
            rr = g->host[0];
            if (!std::isfinite(rr)) return set_err(h, ODWF_EBREAKDOWN, "non-finite GCR residual");
            timed_out = o.max_seconds > 0.0 && elapsed() > o.max_seconds;
        }
        ++cycles;
        if ((rc = launch_axpy_to64(h, 1.0, g->e, ST_FLOAT, nullptr, (double*)w.x_e, st))) return rc;
        if ((rc = residual64(h, c, w.bh, w.x_e, w.t64, w.r64, 3, st))) return rc;
        if ((rc = read_state(h, st))) return rc;
        rr64 = h->state_host->result[3];
        if (!std::isfinite(rr64)) return set_err(h, ODWF_EBREAKDOWN, "non-finite residual");
    }
    double res = 0.0;
    if ((rc = schur_finish(h, c, x, bnorm2, &res, st))) return rc;
    if ((rc = check_fault(h, st))) return rc;
    if (stats) {
        stats->iters = iters;
        stats->reliable_updates = cycles;
        stats->true_residual = res;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!(res <= o.tol))
        return set_err(h, timed_out ? ODWF_ETIMEOUT : ODWF_ENOCONV,
                       timed_out ? "GCR solve stopped at max_seconds" : "GCR solve did not reach tol");
    return ODWF_OK;
}
