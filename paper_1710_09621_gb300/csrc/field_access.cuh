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

// Fifth-dimension mixing of one site's Ns rows staged in shared memory:
// out_k = sum_{s'} M_c[s][s'] w_{s'}k, with c = P_+ for k < 12 and P_- for k >= 12; mt holds the two
// matrices transposed (mt[s' Ns + s] for P_+, then P_-).
template <typename R>
__device__ __forceinline__ void s_mix(const R* mt, const R* sh_site, int s, int Ns, R* out, bool accumulate) {
    R acc[24];
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = 0;
    const int NN = Ns * Ns;
    for (int sp = 0; sp < Ns; ++sp) {
        const R cp = mt[sp * Ns + s];
        const R cm = mt[NN + sp * Ns + s];
        const R* w = sh_site + sp * 24;
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

}  // namespace odwf
