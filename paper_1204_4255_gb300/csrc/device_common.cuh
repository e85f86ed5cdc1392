// device_common.cuh -- complex arithmetic, Philox4x32-10 and Box-Muller on the
// device, shared by every RK4IP kernel of the library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace xsde {

template <typename R> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename R> using cx = typename cplx_of<R>::type;

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulconj(V a, V b) {
    return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// x * (hi + lo) for a factor stored as an FP32 pair whose sum carries ~46 bits.
// The small lo products are formed first and the hi products are added to them
// by FMA, so each component is rounded once with the full factor; adding the lo
// part to an already rounded product would be lost (it is below half an ulp).
// FP64 tables have lo = 0 and use the plain product.
__device__ __forceinline__ float2 cmul_hilo(float2 x, float2 hi, float2 lo) {
    const float tx = fmaf(x.x, lo.x, -x.y * lo.y);
    const float ty = fmaf(x.x, lo.y, x.y * lo.x);
    return make_float2(fmaf(x.x, hi.x, fmaf(-x.y, hi.y, tx)), fmaf(x.x, hi.y, fmaf(x.y, hi.x, ty)));
}
// x * conj(hi + lo), same ordering
__device__ __forceinline__ float2 cmulconj_hilo(float2 x, float2 hi, float2 lo) {
    const float tx = fmaf(x.x, lo.x, x.y * lo.y);
    const float ty = fmaf(x.y, lo.x, -x.x * lo.y);
    return make_float2(fmaf(x.x, hi.x, fmaf(x.y, hi.y, tx)), fmaf(x.y, hi.x, fmaf(-x.x, hi.y, ty)));
}
__device__ __forceinline__ double2 cmul_hilo(double2 x, double2 hi, double2) { return cmul(x, hi); }
__device__ __forceinline__ double2 cmulconj_hilo(double2 x, double2 hi, double2) { return cmulconj(x, hi); }

// a + s*b
template <typename V> __device__ __forceinline__ V caxpy(V a, decltype(V::x) s, V b) {
    return mk<V>(a.x + s * b.x, a.y + s * b.y);
}
template <typename V> __device__ __forceinline__ decltype(V::x) cabs2(V a) { return a.x * a.x + a.y * a.y; }

// complex64: one packed (2 x FP32) instruction per complex add, subtract and
// axpy (sm_100-family FADD2/FFMA2); a - b is b * (-1) + a, rounded once, i.e.
// exactly the FP32 difference
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 caxpy(float2 a, float s, float2 b) { return __ffma2_rn(make_float2(s, s), b, a); }
// i*a and -i*a
template <typename V> __device__ __forceinline__ V cmul_i(V a) { return mk<V>(-a.y, a.x); }
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return mk<V>(a.y, -a.x); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the Weyl key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c.x), lo0 = m0 * c.x;
        uint32_t hi1 = __umulhi(m1, c.z), lo1 = m1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Standard normal pair from the Philox words of counter (point, path, step+1, 0).
template <typename R> struct BoxMuller;
template <> struct BoxMuller<double> {
    __device__ __forceinline__ static double2 pair(uint32_t x0, uint32_t x1) {
        const double s = 2.3283064365386963e-10;        // 2^-32
        double u0 = ((double)x0 + 0.5) * s, u1 = ((double)x1 + 0.5) * s;
        double r = sqrt(-2.0 * log(u0));
        double sn, cs;
        sincospi(2.0 * u1, &sn, &cs);
        return make_double2(r * cs, r * sn);
    }
};
template <> struct BoxMuller<float> {
    __device__ __forceinline__ static float2 pair(uint32_t x0, uint32_t x1) {
        const float s = 2.3283064365386963e-10f, h = 1.1641532182693481e-10f;  // 2^-32, 2^-33
        float u0 = fmaf(__uint2float_rn(x0), s, h), u1 = fmaf(__uint2float_rn(x1), s, h);
        float r = sqrtf(-2.0f * logf(u0));
        float sn, cs;
        sincospif(2.0f * u1, &sn, &cs);
        return make_float2(r * cs, r * sn);
    }
};

template <typename R>
__device__ __forceinline__ cx<R> wiener_pair(uint2 key, uint32_t point, uint32_t path, uint32_t step) {
    uint4 x = philox4x32_10(make_uint4(point, path, step + 1u, 0u), key);
    return BoxMuller<R>::pair(x.x, x.y);
}

}  // namespace xsde
