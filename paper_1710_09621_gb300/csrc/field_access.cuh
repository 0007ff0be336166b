// Device-side access to the internal even-odd chunked fields and links, for the three storage
// precisions. Included by every .cu file of the library.
#pragma once

#include "odwf_internal.h"

namespace odwf {

template <int ST>
struct Store;

// FP64: 12 chunks of one complex (double2) per (cb, s)
template <>
struct Store<ST_DOUBLE> {
    using R = double;
    static constexpr int NCH = 12;
    static __device__ __forceinline__ void load(const void* base, const float*, size_t cb, int s, int Ns,
                                                double v[24]) {
        const double2* p = reinterpret_cast<const double2*>(base) + cb * NCH * Ns + s;
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            double2 c = __ldg(p + (size_t)j * Ns);
            v[2 * j] = c.x;
            v[2 * j + 1] = c.y;
        }
    }
    static __device__ __forceinline__ void store(void* base, float*, size_t cb, int s, int Ns,
                                                 const double v[24]) {
        double2* p = reinterpret_cast<double2*>(base) + cb * NCH * Ns + s;
#pragma unroll
        for (int j = 0; j < NCH; ++j) p[(size_t)j * Ns] = make_double2(v[2 * j], v[2 * j + 1]);
    }
};

// FP32: 6 chunks of two complex (float4) per (cb, s)
template <>
struct Store<ST_FLOAT> {
    using R = float;
    static constexpr int NCH = 6;
    static __device__ __forceinline__ void load(const void* base, const float*, size_t cb, int s, int Ns,
                                                float v[24]) {
        const float4* p = reinterpret_cast<const float4*>(base) + cb * NCH * Ns + s;
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            float4 c = __ldg(p + (size_t)j * Ns);
            v[4 * j] = c.x;
            v[4 * j + 1] = c.y;
            v[4 * j + 2] = c.z;
            v[4 * j + 3] = c.w;
        }
    }
    static __device__ __forceinline__ void store(void* base, float*, size_t cb, int s, int Ns,
                                                 const float v[24]) {
        float4* p = reinterpret_cast<float4*>(base) + cb * NCH * Ns + s;
#pragma unroll
        for (int j = 0; j < NCH; ++j) p[(size_t)j * Ns] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
};

// FP16: 3 chunks of four complex (8 halves in a uint4) per (cb, s), value = half * scale(cb, s)
template <>
struct Store<ST_HALF> {
    using R = float;
    static constexpr int NCH = 3;
    static __device__ __forceinline__ void load(const void* base, const float* scale, size_t cb, int s, int Ns,
                                                float v[24]) {
        const uint4* p = reinterpret_cast<const uint4*>(base) + cb * NCH * Ns + s;
        const float sc = __ldg(scale + cb * Ns + s);
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            uint4 c = __ldg(p + (size_t)j * Ns);
            const __half2* hh = reinterpret_cast<const __half2*>(&c);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float2 f = __half22float2(hh[q]);
                v[8 * j + 2 * q] = f.x * sc;
                v[8 * j + 2 * q + 1] = f.y * sc;
            }
        }
    }
    static __device__ __forceinline__ void store(void* base, float* scale, size_t cb, int s, int Ns,
                                                 const float v[24]) {
        float mx = 0.f;
#pragma unroll
        for (int k = 0; k < 24; ++k) mx = fmaxf(mx, fabsf(v[k]));
        const float sc = mx > 0.f ? mx : 1.f;
        const float inv = 1.f / sc;
        uint4* p = reinterpret_cast<uint4*>(base) + cb * NCH * Ns + s;
#pragma unroll
        for (int j = 0; j < NCH; ++j) {
            uint4 c;
            __half2* hh = reinterpret_cast<__half2*>(&c);
#pragma unroll
            for (int q = 0; q < 4; ++q) hh[q] = __floats2half2_rn(v[8 * j + 2 * q] * inv, v[8 * j + 2 * q + 1] * inv);
            p[(size_t)j * Ns] = c;
        }
        scale[cb * Ns + s] = sc;
    }
};

// Links: FP64 [Vh][8][18] doubles; FP32 and FP16 storage use FP32 links [Vh][8][20] floats.
template <int ST>
struct Links;

template <>
struct Links<ST_DOUBLE> {
    static constexpr int STRIDE = 18;
    static __device__ __forceinline__ void load(const void* base, int cb, int dir, double u[18]) {
        const double2* p = reinterpret_cast<const double2*>(base) + ((size_t)cb * 8 + dir) * 9;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            double2 c = __ldg(p + i);
            u[2 * i] = c.x;
            u[2 * i + 1] = c.y;
        }
    }
};

template <>
struct Links<ST_FLOAT> {
    static constexpr int STRIDE = 20;
    static __device__ __forceinline__ void load(const void* base, int cb, int dir, float u[18]) {
        const float4* p = reinterpret_cast<const float4*>(base) + ((size_t)cb * 8 + dir) * 5;
        float t[20];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            float4 c = __ldg(p + i);
            t[4 * i] = c.x;
            t[4 * i + 1] = c.y;
            t[4 * i + 2] = c.z;
            t[4 * i + 3] = c.w;
        }
#pragma unroll
        for (int i = 0; i < 18; ++i) u[i] = t[i];
    }
};

template <>
struct Links<ST_HALF> : Links<ST_FLOAT> {};

// Two-row links (FP32 [Vh][8][12]): the first two rows of an SU(3) matrix V, whose third row is the
// complex conjugate of the cross product of the first two (V^{-1} = V^dag and det V = 1 make row 2 the
// conjugated cofactors of rows 0 and 1). link12_complete fills u[12..17] = conj(row 0 x row 1) from
// u[0..11]; link12_load reads rows 0 and 1 of link (cb, dir) and completes them.
__device__ __forceinline__ void link12_complete(float u[18]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = (k + 1) % 3, j = (k + 2) % 3;
        const float ar = u[2 * i], ai = u[2 * i + 1], br = u[6 + 2 * j], bi = u[6 + 2 * j + 1];
        const float cr = u[2 * j], ci = u[2 * j + 1], dr = u[6 + 2 * i], di = u[6 + 2 * i + 1];
        // (r0 x r1)_k = r0_i r1_j - r0_j r1_i
        const float re = fmaf(ar, br, -ai * bi) - fmaf(cr, dr, -ci * di);
        const float im = fmaf(ar, bi, ai * br) - fmaf(cr, di, ci * dr);
        u[12 + 2 * k] = re;
        u[13 + 2 * k] = -im;
    }
}

__device__ __forceinline__ void link12_load(const float* base, int cb, int dir, float u[18]) {
    const float4* p = reinterpret_cast<const float4*>(base) + ((size_t)cb * 8 + dir) * 3;
    const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    u[0] = a.x, u[1] = a.y, u[2] = a.z, u[3] = a.w;
    u[4] = b.x, u[5] = b.y, u[6] = b.z, u[7] = b.w;
    u[8] = c.x, u[9] = c.y, u[10] = c.z, u[11] = c.w;
    link12_complete(u);
}

// Rows of 24 reals (one (site, s) spinor) in shared memory, moved as 16-byte vectors. Every row
// start is 16-byte aligned: rows are 96 (FP32) or 192 (FP64) bytes and the staging buffers start at
// 16-byte aligned offsets.
__device__ __forceinline__ void row24_store(float* dst, const float* v) {
#pragma unroll
    for (int q = 0; q < 6; ++q)
        reinterpret_cast<float4*>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}
__device__ __forceinline__ void row24_store(double* dst, const double* v) {
#pragma unroll
    for (int q = 0; q < 12; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(v[2 * q], v[2 * q + 1]);
}
__device__ __forceinline__ void row4_load(const float* p, float* o) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = t.x, o[1] = t.y, o[2] = t.z, o[3] = t.w;
}
__device__ __forceinline__ void row4_load(const double* p, double* o) {
    const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
    o[0] = t0.x, o[1] = t0.y, o[2] = t1.x, o[3] = t1.y;
}

// Row stride (in reals) of the padded staging rows of the FMA fifth-dimension mixing: 28 floats
// (112 bytes) or 26 doubles (208 bytes) put the 16-byte row stores of 8 consecutive lanes on 8
// distinct 4-bank groups, where the unpadded 96 / 192-byte rows collide two- and four-way.
template <typename R>
constexpr int kRowStride = sizeof(R) == 4 ? 28 : 26;

// Fifth-dimension mixing of one site's Ns rows staged in shared memory (row stride rs reals):
// out_k = sum_{s'} M_c[s][s'] w_{s'}k, with c = P_+ for k < 12 and P_- for k >= 12; mt holds the two
// matrices transposed (mt[s' Ns + s] for P_+, then P_-).
template <typename R>
__device__ __forceinline__ void s_mix(const R* mt, const R* sh_site, int s, int Ns, R* out, bool accumulate,
                                      int rs = 24) {
    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    const int NN = Ns * Ns;
    for (int sp = 0; sp < Ns; ++sp) {
        const R cp = mt[sp * Ns + s];
        const R cm = mt[NN + sp * Ns + s];
        const R* w = sh_site + sp * rs;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            R t[4];
            row4_load(w + 4 * q, t);
            const R c = q < 3 ? cp : cm;
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[4 * q + i] = fma(c, t[i], acc[4 * q + i]);
        }
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) out[k] = accumulate ? out[k] + acc[k] : acc[k];
}

// As s_mix, with the two chiralities' transposed matrices interleaved, mp[2 (s' Ns + s)] = M_+[s][s']
// and mp[2 (s' Ns + s) + 1] = M_-[s][s'], so that one 8- (FP32) or 16-byte (FP64) load per s' fetches
// both coefficients.
__device__ __forceinline__ void coef_pair(const float* mp, int i, float& cp, float& cm) {
    const float2 c = reinterpret_cast<const float2*>(mp)[i];
    cp = c.x, cm = c.y;
}
__device__ __forceinline__ void coef_pair(const double* mp, int i, double& cp, double& cm) {
    const double2 c = reinterpret_cast<const double2*>(mp)[i];
    cp = c.x, cm = c.y;
}
template <typename R>
__device__ __forceinline__ void s_mix2(const R* mp, const R* sh_site, int s, int Ns, R* out, bool accumulate,
                                       int rs) {
    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    for (int sp = 0; sp < Ns; ++sp) {
        R cp, cm;
        coef_pair(mp, sp * Ns + s, cp, cm);
        const R* w = sh_site + sp * rs;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            R t[4];
            row4_load(w + 4 * q, t);
            const R c = q < 3 ? cp : cm;
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[4 * q + i] = fma(c, t[i], acc[4 * q + i]);
        }
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) out[k] = accumulate ? out[k] + acc[k] : acc[k];
}

// ---- structured fifth-dimension products (see SStruct), Ns = kStructNs ----------------------------
// After the hop, each (site, s) thread stores its 24-real row; then the thread of slice j < 12 of
// the site takes complex component j of all Ns rows (one column, re and im), applies A or A^{-1}
// of that component's chirality by the O(Ns) recurrence in registers, and writes the column back;
// finally every thread reads its own row again. The coefficients are indexed by the step of the
// recurrence only (compile-time, unrolled), so in a kernel whose arguments are the SStruct by value
// they are constant-bank operands of the FMAs.
template <typename R>
__device__ __forceinline__ const SStructT<R>& sst_of(const SStruct& s);
template <>
__device__ __forceinline__ const SStructT<float>& sst_of<float>(const SStruct& s) { return s.f; }
template <>
__device__ __forceinline__ const SStructT<double>& sst_of<double>(const SStruct& s) { return s.d; }

// Shared-memory geometry of the structured staging rows: row stride kSRow reals, site stride kSSite
// reals. With 28-float rows the 16-byte row stores of 8 consecutive slices hit 8 distinct 4-bank
// groups, and the column loads of one site (a half-warp: 12 lanes reading the 24 reals of one row)
// hit 24 distinct banks.
template <typename R>
constexpr int kSRow = sizeof(R) == 4 ? 28 : 26;
template <typename R>
constexpr int kSSite = kStructNs * kSRow<R> + (sizeof(R) == 4 ? 16 : 4);

__device__ __forceinline__ void pair_ld(const float* p, float& a, float& b) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    a = t.x, b = t.y;
}
__device__ __forceinline__ void pair_ld(const double* p, double& a, double& b) {
    const double2 t = *reinterpret_cast<const double2*>(p);
    a = t.x, b = t.y;
}
__device__ __forceinline__ void pair_st(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void pair_st(double* p, double a, double b) {
    *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// A^{-1} = W (1 + L) B^{-1} W on one complex column (x = xr + i xi) in recurrence order:
//   p_0 = 0, p_s = (omega_s^{1/2}/d_s) x_s - (e_s/d_s) p_{s-1};  B y = W x with y_s = p_s + q_s u,
//   u = y_0 = (omega_0^{1/2} x_0 + m e_0 p_{N-1}) / (d_0 - m e_0 q_{N-1});
//   out_s = omega_s^{1/2} (y_s + y_{s-1}) (s >= 1),  out_0 = omega_0^{1/2} (y_0 - m y_{N-1}).
template <typename R, int N>
__device__ __forceinline__ void s_ainv_col(const SStructT<R>& k, int c, R* xr, R* xi) {
    const R z0r = k.w[0] * xr[0], z0i = k.w[0] * xi[0];
    xr[0] = 0, xi[0] = 0;
#pragma unroll
    for (int s = 1; s < N; ++s) {
        xr[s] = fma(-k.f[s], xr[s - 1], k.rw[s] * xr[s]);
        xi[s] = fma(-k.f[s], xi[s - 1], k.rw[s] * xi[s]);
    }
    const R me0 = c ? k.me0[1] : k.me0[0], cu = c ? k.cu[1] : k.cu[0], m = c ? k.m[1] : k.m[0];
    const R ur = cu * fma(me0, xr[N - 1], z0r), ui = cu * fma(me0, xi[N - 1], z0i);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        xr[s] = fma(k.q[s], ur, xr[s]);
        xi[s] = fma(k.q[s], ui, xi[s]);
    }
    const R ylr = xr[N - 1], yli = xi[N - 1];
#pragma unroll
    for (int s = N - 1; s >= 1; --s) {
        xr[s] = k.w[s] * (xr[s] + xr[s - 1]);
        xi[s] = k.w[s] * (xi[s] + xi[s - 1]);
    }
    xr[0] = k.w[0] * fma(-m, ylr, xr[0]);
    xi[0] = k.w[0] * fma(-m, yli, xi[0]);
}

// A = (4 - m0 - 1/omega) + 2 W^{-1} (1 + L)^{-1} W^{-1} on one complex column in recurrence order:
//   z = W^{-1} x, p_0 = 0, p_s = z_s - p_{s-1}, (1 + L)^{-1} z = p + (-1)^s u, u = (z_0 + m p_{N-1})/(1 + m).
template <typename R, int N>
__device__ __forceinline__ void s_a_col(const SStructT<R>& k, int c, R* xr, R* xi) {
    const R z0r = k.wi[0] * xr[0], z0i = k.wi[0] * xi[0];
    R pr = 0, pi = 0;
    xr[0] = k.adiag[0] * xr[0], xi[0] = k.adiag[0] * xi[0];
#pragma unroll
    for (int s = 1; s < N; ++s) {
        pr = fma(k.wi[s], xr[s], -pr);
        pi = fma(k.wi[s], xi[s], -pi);
        xr[s] = fma(k.wi[s], pr + pr, k.adiag[s] * xr[s]);
        xi[s] = fma(k.wi[s], pi + pi, k.adiag[s] * xi[s]);
    }
    const R m = c ? k.m[1] : k.m[0], au = c ? k.au[1] : k.au[0];
    const R ur = au * fma(m, pr, z0r), ui = au * fma(m, pi, z0i);
#pragma unroll
    for (int s = 0; s < N; ++s) {
        xr[s] = fma(k.wi2s[s], ur, xr[s]);
        xi[s] = fma(k.wi2s[s], ui, xi[s]);
    }
}

// in-register reversal of the s order of one column (a per-lane select, so that every lane can load
// and store its rows in the same order)
template <typename R, int N>
__device__ __forceinline__ void col_reverse(bool rev, R* x) {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
        const R a = x[i], b = x[N - 1 - i];
        x[i] = rev ? b : a;
        x[N - 1 - i] = rev ? a : b;
    }
}

// The column pass of thread j of one site (site: its staged rows, row stride rs); threads j >= 12
// have no column. P_+ components (j < 6) run forward in s and P_- ones backward, both reversed for
// a transposed operator. All lanes load and store the rows in s order (the P_+ and P_- columns of a
// site then lie in one row, on distinct banks) and the reversed lanes flip their registers instead.
template <typename R, int N>
__device__ __forceinline__ void s_struct_col(const SStruct& sc, int sop, R* site, int rs, int j) {
    if (j >= 12) return;
    const SStructT<R>& k = sst_of<R>(sc);
    const int c = j < 6 ? 0 : 1;
    const bool rev = (c == 1) != ((sop & SOP_T) != 0);
    R* p0 = site + 2 * j;
    R xr[N], xi[N];
#pragma unroll
    for (int q = 0; q < N; ++q) pair_ld(p0 + q * rs, xr[q], xi[q]);
    col_reverse<R, N>(rev, xr);
    col_reverse<R, N>(rev, xi);
    if ((sop & 3) == SOP_AINV) s_ainv_col<R, N>(k, c, xr, xi);
    else s_a_col<R, N>(k, c, xr, xi);
    col_reverse<R, N>(rev, xr);
    col_reverse<R, N>(rev, xi);
#pragma unroll
    for (int q = 0; q < N; ++q) pair_st(p0 + q * rs, xr[q], xi[q]);
}

// out = [out +] the staged row at p (24 reals, 16-byte aligned)
template <typename R>
__device__ __forceinline__ void row24_load(const R* p, R* out, bool accumulate) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        R t[4];
        row4_load(p + 4 * q, t);
#pragma unroll
        for (int i = 0; i < 4; ++i) out[4 * q + i] = accumulate ? out[4 * q + i] + t[i] : t[i];
    }
}

// ---- fifth-dimension mixing on the tensor cores, Ns = 16 -----------------------------------------
// With Ns = 16 a warp holds exactly two sites (its own 32 (site, s) threads), so the mixing of those
// two sites is warp-local: per chirality c the product D = A_c B of the 16 x 16 matrix A_c with the
// 16 x 24 block B (rows s, columns = 12 components of chirality c of the two sites) is three m16n8k8
// TF32 tiles, two k-steps each. FP32 accuracy is kept by the split X = X_hi + X_lo into TF32 parts:
// D = A_lo B_hi + A_hi B_lo + A_hi B_hi (the A_lo B_lo term, of relative size 2^-22, is dropped).
// The A fragments (hi and lo) of both chiralities are built once per CTA (s_mix16_afrag); D is
// written back in place over the staged rows (chirality c only reads and writes components
// 12 c .. 12 c + 11) and each thread then reads its own row.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// uint32 entries of the fragment table: [chirality 2][k-step 2][hi, lo][lane 32][4] (a lane's 16-byte
// reads of one table are consecutive: conflict-free)
constexpr int kAfrag16Words = 2 * 2 * 32 * 8;

// Fragment table from the transposed matrix pair mt (A_c[s_out][s_in] = mt[c 256 + s_in 16 + s_out]);
// every thread of the CTA takes a share; the caller synchronises the CTA afterwards.
__device__ __forceinline__ void s_mix16_afrag(const double* mt, uint32_t* afr, int tid, int nth) {
    for (int e = tid; e < kAfrag16Words / 2; e += nth) {
        const int j = e & 3, lane = (e >> 2) & 31, ks = (e >> 7) & 1, c = e >> 8;
        const int gid = lane >> 2, tig = lane & 3;
        const int row = gid + ((j & 1) ? 8 : 0), col = ks * 8 + tig + ((j & 2) ? 4 : 0);
        const float x = (float)mt[c * 256 + col * 16 + row];
        const uint32_t hi = tf32_rna(x);
        uint32_t* w = afr + ((c * 2 + ks) * 2 * 32 + lane) * 4 + j;
        w[0] = hi;
        w[32 * 4] = tf32_rna(x - __uint_as_float(hi));
    }
}

// Collective over the warp (all 32 lanes), after the warp's rows are staged in sh and a __syncwarp:
// out = [out +] (mixed row of this thread). sh rows are [site][s][24] with Ns = 16.
__device__ __forceinline__ void s_mix16_tc(const uint32_t* afr, float* sh, int lane, int warp, int row,
                                           float* out, bool accumulate) {
    const int gid = lane >> 2, tig = lane & 3;
    float* base = sh + (size_t)warp * 2 * 16 * 24;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        float acc[3][4];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
            const int col = 8 * q + gid;
            const float* bp = base + (col >= 12 ? 16 * 24 + col - 12 : col) + c * 12;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const uint4* ap = reinterpret_cast<const uint4*>(afr + ((c * 2 + ks) * 2 * 32 + lane) * 4);
                const uint4 h4 = ap[0], l4 = ap[32];
                const uint32_t ah[4] = {h4.x, h4.y, h4.z, h4.w}, al[4] = {l4.x, l4.y, l4.z, l4.w};
                const float b0 = bp[(ks * 8 + tig) * 24], b1 = bp[(ks * 8 + tig + 4) * 24];
                uint32_t bh[2], bl[2];
                bh[0] = tf32_rna(b0);
                bh[1] = tf32_rna(b1);
                bl[0] = tf32_rna(b0 - __uint_as_float(bh[0]));
                bl[1] = tf32_rna(b1 - __uint_as_float(bh[1]));
                mma_tf32(acc[q], al, bh);
                mma_tf32(acc[q], ah, bl);
                mma_tf32(acc[q], ah, bh);
            }
        }
        __syncwarp();  // every lane has read chirality c's components before they are overwritten
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int col = 8 * q + 2 * tig;  // even: (col, col + 1) stay within one site
            float* d0 = base + (col >= 12 ? 16 * 24 + col - 12 : col) + c * 12 + gid * 24;
            *reinterpret_cast<float2*>(d0) = make_float2(acc[q][0], acc[q][1]);
            *reinterpret_cast<float2*>(d0 + 8 * 24) = make_float2(acc[q][2], acc[q][3]);
        }
    }
    __syncwarp();
    const float* r = sh + (size_t)row * 24;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float t[4];
        row4_load(r + 4 * q, t);
#pragma unroll
        for (int i = 0; i < 4; ++i) out[4 * q + i] = accumulate ? out[4 * q + i] + t[i] : t[i];
    }
}

}  // namespace odwf
