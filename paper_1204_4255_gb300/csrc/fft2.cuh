// fft2.cuh -- two-stage register FFTs for warp-owned columns (sm_103a).
//
// A length-N transform is carried by P lanes of one warp (P = 8 or 16); lane
// t holds the E = N/P elements x[t + P m], m = 0..E-1, in registers.  The
// transform is one radix-E stage (a whole DFT_E in registers, no twiddles),
// one exchange through the column's shared-memory slots, and E/P radix-P
// butterflies with the twiddles w_N^(r j) -- the Stockham autosort of
// fft.cuh with only two stages, so only one exchange and only __syncwarp():
//   stage 1 (Ns = 1, radix E) : butterfly j = t, inputs x[t + P r], outputs y[E t + r]
//   stage 2 (Ns = E, radix P) : butterflies j = t + P q (q < E/P), inputs x[j + E r],
//                               twiddles w^(r j), outputs y[j + E r] -- natural order.
// Forward transforms (S = -1) are unnormalised, inverse ones (S = +1) take the
// conjugate roots (XMDS2 Sec. 2.2's spectral transform for the Fourier basis
// of Sec. 2.1).  The radix-16 and radix-32 DFTs are 4 x 4 and 4 x 8 products
// whose internal roots are compile-time FP64 values split into an FP32 pair
// and applied with the compensated products of device_common.cuh.
#pragma once

#include <type_traits>

#include "fft.cuh"

namespace xsde {

// cos and sin of 2 pi k / n in FP64, evaluated at compile time: the angle is
// reduced to the nearest quadrant (|r| <= pi/4, exact integer numerator) and
// the Taylor series of r is summed far past double precision.
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, s = x;
    for (int i = 1; i < 14; ++i) {
        term *= -x * x / ((2.0 * i) * (2.0 * i + 1.0));
        s += term;
    }
    return s;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, s = 1.0;
    for (int i = 1; i < 14; ++i) {
        term *= -x * x / ((2.0 * i - 1.0) * (2.0 * i));
        s += term;
    }
    return s;
}
__host__ __device__ constexpr double cos_2pi_frac(int k, int n) {
    k = ((k % n) + n) % n;
    const int q = (8 * k + n) / (2 * n);   // nearest multiple of pi/2
    const double r = 6.283185307179586476925286766559 * (double)(4 * k - q * n) / (4.0 * n);
    return (q & 3) == 0 ? taylor_cos(r) : (q & 3) == 1 ? -taylor_sin(r) : (q & 3) == 2 ? -taylor_cos(r) : taylor_sin(r);
}
__host__ __device__ constexpr double sin_2pi_frac(int k, int n) {
    k = ((k % n) + n) % n;
    const int q = (8 * k + n) / (2 * n);
    const double r = 6.283185307179586476925286766559 * (double)(4 * k - q * n) / (4.0 * n);
    return (q & 3) == 0 ? taylor_sin(r) : (q & 3) == 1 ? taylor_cos(r) : (q & 3) == 2 ? -taylor_sin(r) : -taylor_cos(r);
}

// compile-time loop: f(std::integral_constant<int, i>) for i in [B, E)
template <int B, int E, typename F> __device__ __forceinline__ void static_for(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// x * exp(S 2 pi i K / N) for compile-time K, N.  Multiples of pi/2 are exact
// swaps and sign changes; odd multiples of pi/4 use the split 1/sqrt(2) of
// dft8; every other root is an FP32 hi + lo pair of the FP64 value.
template <int K, int N, int S> __device__ __forceinline__ float2 rot_const(float2 x) {
    constexpr int k = ((K % N) + N) % N;
    constexpr int e8 = (8 * k) % N == 0 ? (8 * k) / N : -1;   // k = e8 N / 8
    if constexpr (k == 0) {
        return x;
    } else if constexpr (e8 >= 0) {
        // exp(S i pi e8 / 4): (S < 0) e8 -> 8 - e8 with S > 0
        constexpr int e = S < 0 ? (8 - e8) % 8 : e8;
        if constexpr (e == 2) return cmul_i(x);
        else if constexpr (e == 4) return make_float2(-x.x, -x.y);
        else if constexpr (e == 6) return cmul_mi(x);
        else if constexpr (e == 1) return make_float2(mul_rsqrt2(x.x - x.y), mul_rsqrt2(x.x + x.y));
        else if constexpr (e == 3) return make_float2(-mul_rsqrt2(x.x + x.y), mul_rsqrt2(x.x - x.y));
        else if constexpr (e == 5) return make_float2(mul_rsqrt2(x.y - x.x), -mul_rsqrt2(x.x + x.y));
        else return make_float2(mul_rsqrt2(x.x + x.y), mul_rsqrt2(x.y - x.x));   // e == 7
    } else {
        constexpr double c = cos_2pi_frac(k, N), s = S * sin_2pi_frac(k, N);
        constexpr float ch = (float)c, sh = (float)s;
        constexpr float cl = (float)(c - (double)ch), sl = (float)(s - (double)sh);
        return cmul_hilo(x, make_float2(ch, sh), make_float2(cl, sl));
    }
}

// DFT of R = 16 or 32 points in registers, natural order in and out:
// n = n1 + 4 n2, k = k2 + (R/4) k1; inner DFT_{R/4} over n2, roots w_R^(n1 k2),
// outer DFT_4 over n1.
template <int R, int S> __device__ __forceinline__ void dft_4x(float2 *u) {
    constexpr int Q = R / 4;
    static_for<0, 4>([&](auto n1c) {
        constexpr int n1 = decltype(n1c)::value;
        float2 v[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) v[n2] = u[n1 + 4 * n2];
        dft<Q, S>(v);
        static_for<0, Q>([&](auto k2c) {
            constexpr int k2 = decltype(k2c)::value;
            u[n1 + 4 * k2] = rot_const<n1 * k2, R, S>(v[k2]);
        });
    });
    float2 o[R];
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
        float2 v[4] = {u[4 * k2], u[4 * k2 + 1], u[4 * k2 + 2], u[4 * k2 + 3]};
        dft4<S>(v);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) o[k2 + Q * k1] = v[k1];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) u[k] = o[k];
}

template <int R, int S> __device__ __forceinline__ void dft_reg(float2 *u) {
    if constexpr (R <= 8) dft<R, S>(u);
    else dft_4x<R, S>(u);
}

// Physical row of logical index i during a column exchange: the low three bits
// are XOR-ed with the three bits above log2(E).  With swizzled tile rows (two
// or four columns per warp) both the stage-1 writes and the stage-2 reads then
// spread a column's lanes evenly over the eight 16-byte bank groups.
template <int E> __device__ __forceinline__ int xslot(int i) { return i ^ ((i >> ilog2c(E)) & 7); }

// Twiddle table of the two-stage plan: entry (r - 1) E + j holds w_N^(r j)
// for r in [1, P), j in [0, E) as (cos_hi, sin_hi, cos_lo, sin_lo).
template <int N, int E> __host__ __device__ constexpr int warp_fft_table_size() { return (N / E - 1) * E; }

// One transform of the line held by this lane's group of P lanes.  `xat(i)` is
// the address of the exchange slot of logical index i (the caller's layout
// spreads both exchange patterns over the banks); the caller has synchronised
// the warp since the slots were last read.  Ends with a __syncwarp() before the
// result is in registers, so the slots may be rewritten by the caller.
template <int N, int E, int S, typename XAt, typename Tw>
__device__ __forceinline__ void warp_fft(float2 (&x)[E], int t, const XAt &xat, const Tw &tw) {
    constexpr int P = N / E;
    static_assert(P == 8 || P == 16, "two-stage plan: 8 or 16 lanes per line");
    static_assert(E >= P && E % P == 0, "two-stage plan: E >= P");
    dft_reg<E, S>(x);
#pragma unroll
    for (int r = 0; r < E; ++r) *xat(E * t + r) = x[r];
    __syncwarp();
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = *xat(t + P * m);
    __syncwarp();
#pragma unroll
    for (int q = 0; q < E / P; ++q) {
        const int j = t + P * q;
        float2 u[P];
        u[0] = x[q];
#pragma unroll
        for (int r = 1; r < P; ++r) u[r] = twiddle_mul<S>(x[q + (E / P) * r], tw((r - 1) * E + j));
        dft_reg<P, S>(u);
#pragma unroll
        for (int r = 0; r < P; ++r) x[q + (E / P) * r] = u[r];
    }
}

// The conjugate transpose of warp_fft<N, E, -1>: stage 2 transposed (DFT_P with
// the conjugate roots, then the conjugate twiddles), the exchange transposed,
// then DFT_E with the conjugate roots.  In exact arithmetic it is N times the
// inverse of the forward transform computed with the same rounded twiddles, so
// a forward / inverse pair around a unit-modulus factor is unitary whatever the
// twiddles' rounding, where the same-order inverse warp_fft<N, E, +1> is not
// (on the 512^2 GPE over 2000 steps the norm drifts half as much).  Same
// synchronisation contract as warp_fft.
template <int N, int E, typename XAt, typename Tw>
__device__ __forceinline__ void warp_ifft_t(float2 (&x)[E], int t, const XAt &xat, const Tw &tw) {
    constexpr int P = N / E;
    static_assert(P == 8 || P == 16, "two-stage plan: 8 or 16 lanes per line");
#pragma unroll
    for (int q = 0; q < E / P; ++q) {
        const int j = t + P * q;
        float2 u[P];
#pragma unroll
        for (int r = 0; r < P; ++r) u[r] = x[q + (E / P) * r];
        dft_reg<P, +1>(u);
        x[q] = u[0];
#pragma unroll
        for (int r = 1; r < P; ++r) x[q + (E / P) * r] = twiddle_mul<+1>(u[r], tw((r - 1) * E + j));
    }
#pragma unroll
    for (int m = 0; m < E; ++m) *xat(t + P * m) = x[m];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < E; ++r) x[r] = *xat(E * t + r);
    __syncwarp();
    dft_reg<E, +1>(x);
}

}  // namespace xsde
