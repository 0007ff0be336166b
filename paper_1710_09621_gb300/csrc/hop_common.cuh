// Device building blocks shared by the hopping kernels (kernels.cu, hop_pair.cu): spin projection and
// reconstruction, the SU(3) product of a half spinor, the fused epilogues of the CGNE iteration and the
// deterministic grid reduction behind them.
#pragma once

#include "field_access.cuh"

namespace odwf {

// ---- complex helpers on interleaved real arrays ------------------------------------------------
// spinor index of (spin, color) real part: (spin * 3 + color) * 2

template <typename R>
__device__ __forceinline__ void cadd(R* o, const R* a) { o[0] += a[0]; o[1] += a[1]; }

// h = psi_up + SIGN * B_mu psi_dn  (SIGN = -1 for 1 - gamma_mu, +1 for 1 + gamma_mu)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void project(const R* p, R* h) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R* u0 = p + (0 * 3 + c) * 2;
        const R* u1 = p + (1 * 3 + c) * 2;
        const R* d0 = p + (2 * 3 + c) * 2;
        const R* d1 = p + (3 * 3 + c) * 2;
        R* h0 = h + (0 * 3 + c) * 2;
        R* h1 = h + (1 * 3 + c) * 2;
        if (MU == 0) {  // B = -i sigma_1: (B d)_0 = -i d1, (B d)_1 = -i d0; -i z = (z.im, -z.re)
            h0[0] = u0[0] + SIGN * d1[1]; h0[1] = u0[1] - SIGN * d1[0];
            h1[0] = u1[0] + SIGN * d0[1]; h1[1] = u1[1] - SIGN * d0[0];
        } else if (MU == 1) {  // B = -i sigma_2 = [[0,-1],[1,0]]: (B d)_0 = -d1, (B d)_1 = d0
            h0[0] = u0[0] - SIGN * d1[0]; h0[1] = u0[1] - SIGN * d1[1];
            h1[0] = u1[0] + SIGN * d0[0]; h1[1] = u1[1] + SIGN * d0[1];
        } else if (MU == 2) {  // B = -i sigma_3: (B d)_0 = -i d0, (B d)_1 = +i d1; i z = (-z.im, z.re)
            h0[0] = u0[0] + SIGN * d0[1]; h0[1] = u0[1] - SIGN * d0[0];
            h1[0] = u1[0] - SIGN * d1[1]; h1[1] = u1[1] + SIGN * d1[0];
        } else {  // B = 1
            h0[0] = u0[0] + SIGN * d0[0]; h0[1] = u0[1] + SIGN * d0[1];
            h1[0] = u1[0] + SIGN * d1[0]; h1[1] = u1[1] + SIGN * d1[1];
        }
    }
}

// v_up += w ; v_dn += SIGN * C_mu w   (SIGN = -1 for 1 - gamma_mu, +1 for 1 + gamma_mu)
template <int MU, int SIGN, typename R>
__device__ __forceinline__ void reconstruct(R* v, const R* w) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const R* w0 = w + (0 * 3 + c) * 2;
        const R* w1 = w + (1 * 3 + c) * 2;
        R* v0 = v + (0 * 3 + c) * 2;
        R* v1 = v + (1 * 3 + c) * 2;
        R* v2 = v + (2 * 3 + c) * 2;
        R* v3 = v + (3 * 3 + c) * 2;
        cadd(v0, w0);
        cadd(v1, w1);
        if (MU == 0) {  // C = i sigma_1: (C w)_0 = i w1, (C w)_1 = i w0
            v2[0] += SIGN * (-w1[1]); v2[1] += SIGN * w1[0];
            v3[0] += SIGN * (-w0[1]); v3[1] += SIGN * w0[0];
        } else if (MU == 1) {  // C = i sigma_2 = [[0,1],[-1,0]]: (C w)_0 = w1, (C w)_1 = -w0
            v2[0] += SIGN * w1[0]; v2[1] += SIGN * w1[1];
            v3[0] -= SIGN * w0[0]; v3[1] -= SIGN * w0[1];
        } else if (MU == 2) {  // C = i sigma_3: (C w)_0 = i w0, (C w)_1 = -i w1
            v2[0] += SIGN * (-w0[1]); v2[1] += SIGN * w0[0];
            v3[0] += SIGN * w1[1]; v3[1] += SIGN * (-w1[0]);
        } else {  // C = 1
            v2[0] += SIGN * w0[0]; v2[1] += SIGN * w0[1];
            v3[0] += SIGN * w1[0]; v3[1] += SIGN * w1[1];
        }
    }
}

// w[spin a] = U h[spin a] for the two spins of a half spinor
template <typename R>
__device__ __forceinline__ void su3_mul_half(const R* u, const R* h, R* w) {
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R re = 0, im = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const R ur = u[(i * 3 + j) * 2], ui = u[(i * 3 + j) * 2 + 1];
                const R hr = h[(a * 3 + j) * 2], hi = h[(a * 3 + j) * 2 + 1];
                re = fma(ur, hr, re);
                re = fma(-ui, hi, re);
                im = fma(ur, hi, im);
                im = fma(ui, hr, im);
            }
            w[(a * 3 + i) * 2] = re;
            w[(a * 3 + i) * 2 + 1] = im;
        }
    }
}

template <typename R>
__device__ __forceinline__ void g5_flip(R* v) {
#pragma unroll
    for (int k = 12; k < 24; ++k) v[k] = -v[k];
}


__device__ __forceinline__ double block_reduce_sum(double v, double* wsum) {
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int w = 0; w < nwarps; ++w) tot += wsum[w];
    return tot;  // valid in thread (0,0)
}

// Deterministic grid reduction: every block writes its partial; the last block to finish sums
// the partials in index order and runs the epilogue's scalar update.
template <int EPI>
__device__ void grid_finalize(const HopArgs& a, double part) {
    __shared__ double wsum[32];
    __shared__ int is_last;
    const double bsum = block_reduce_sum(part, wsum);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        a.partials[blockIdx.x] = bsum;
        __threadfence();
        const unsigned t = atomicAdd(&a.state->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nth = blockDim.x * blockDim.y;
    double acc = 0.0;
    for (int i = tid; i < (int)gridDim.x; i += nth) acc += ((volatile double*)a.partials)[i];
    const double tot = block_reduce_sum(acc, wsum);
    if (tid == 0) {
        CGState* st = a.state;
        st->ticket = 0;
        if (EPI == EPI_CG_A) {
            const double rr_new = tot;
            st->iter += 1;
            if (!isfinite(rr_new)) {
                st->flag = FLAG_BREAKDOWN;
            } else {
                st->beta = rr_new / st->rr;
                st->rr = rr_new;
                if (rr_new > st->rr_max) st->rr_max = rr_new;
                if (rr_new <= st->tol2) st->flag = FLAG_CONVERGED;
                else if (st->delta2 > 0.0 && rr_new < st->delta2 * st->rr_max) st->flag = FLAG_UPDATE;
                else if (st->iter >= st->maxiter) st->flag = FLAG_MAXITER;
            }
        } else if (EPI == EPI_CG_B) {
            st->pp = tot;
            if (!(tot > 0.0) || !isfinite(tot)) st->flag = FLAG_BREAKDOWN;
            else st->alpha = st->rr / tot;
        } else {
            st->result[a.slot] = tot;
        }
    }
}

// Epilogue of the fused kernels for one (site, s): store, residual, or the CGNE updates; adds the
// thread's contribution to the block reduction in `part`.
template <int ST, int EPI>
__device__ __forceinline__ void epilogue(const HopArgs& a, int cb, int s, typename Store<ST>::R* v,
                                         const typename Store<ST>::R* ow, double alpha, double beta, double& part) {
    using S = Store<ST>;
    using R = typename S::R;
    const int Ns = a.Ns;
    if (EPI == EPI_STORE || EPI == EPI_STORE_NORM) {
        S::store(a.out, a.out_scale, (size_t)cb, s, Ns, v);
        if (EPI == EPI_STORE_NORM) {
            R t = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) t = fma(v[k], v[k], t);
            part += (double)t;
        }
    } else if (EPI == EPI_RESID) {
        R b[24];
        S::load(a.x, a.x_scale, (size_t)cb, s, Ns, b);
        R t = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            b[k] -= v[k];
            t = fma(b[k], b[k], t);
        }
        S::store(a.out, a.out_scale, (size_t)cb, s, Ns, b);
        part += (double)t;
    } else if (EPI == EPI_CG_A) {
        // x += alpha * own (own = p, without gamma_5), r -= alpha * v
        R x[24], r[24];
        S::load(a.x, a.x_scale, (size_t)cb, s, Ns, x);
        S::load(a.r, a.r_scale, (size_t)cb, s, Ns, r);
        const R al = (R)alpha;
        R t = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            x[k] = fma(al, ow[k], x[k]);
            r[k] = fma(-al, v[k], r[k]);
            t = fma(r[k], r[k], t);
        }
        S::store(a.x, a.x_scale, (size_t)cb, s, Ns, x);
        S::store(a.r, a.r_scale, (size_t)cb, s, Ns, r);
        part += (double)t;
    } else if (EPI == EPI_CG_B) {
        // p = v + beta * p
        R p[24];
        S::load(a.r, a.r_scale, (size_t)cb, s, Ns, p);
        const R be = (R)beta;
        R t = 0;
#pragma unroll
        for (int k = 0; k < 24; ++k) {
            p[k] = fma(be, p[k], v[k]);
            t = fma(p[k], p[k], t);
        }
        S::store(a.r, a.r_scale, (size_t)cb, s, Ns, p);
        part += (double)t;
    }
}

// ---- asynchronous bulk copies into shared memory, completed on an mbarrier ----------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// orders this thread's (and, after a barrier, its warp's) generic-proxy shared-memory accesses before the
// asynchronous-proxy writes of the bulk copies it issues next
__device__ __forceinline__ void fence_proxy_async_cta() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` for at most ~1 s of SM clock (limit <= 0), or for at most `limit` cycles
// polled with the non-blocking test (a caller-set limit, which tests use to make the wait run out);
// false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = 0) {
    const long long t0 = clock64();
    if (limit > 0) {
        while (!mbar_test_wait(bar, parity))
            if (clock64() - t0 > limit) return false;
        return true;
    }
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > 2000000000LL) return false;
    }
    return true;
}

}  // namespace odwf
