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
// The forward transform (XMDS2 Sec. 2.2's spectral transform for the Fourier
// basis of Sec. 2.1) is unnormalised.  The backward one is its exact inverse
// (times N), taken factor by factor in reverse order: every root the forward
// multiplies by is the FP32 rounding w~ of the FP64 value, and the backward
// multiplies by 1/w~ = conj(w~) (1 + eps), eps = 1/|w~|^2 - 1, held as the
// pair conj(w~) + conj(w~) eps and applied with one rounding per component
// (cmulconj_hilo: a correction of a fraction of an ulp added after the product
// had been rounded would be lost, and systematically so).  A forward /
// backward pair is then the identity up to the arithmetic's rounding, whatever
// the modulus of the rounded roots -- the modulus bias of plain FP32 roots in
// both directions drains the norm by ~1e-4 over a 2000-step 2D run -- at 4 + 8
// instructions per root pair instead of 8 + 8 for compensated roots both ways.
// The radix-16 and radix-32 DFTs are 4 x 4 and 4 x 8 products whose internal
// roots are compile-time FP64 values rounded the same way.
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

// The FP32 rounding of exp(-2 pi i K / N) for compile-time K, N, and the eps
// of its exact inverse.
template <int K, int N> struct Root {
    static constexpr int k = ((K % N) + N) % N;
    static constexpr double c = cos_2pi_frac(k, N), s = -sin_2pi_frac(k, N);
    static constexpr float ch = (float)c, sh = (float)s;
    static constexpr double eps = 1.0 / ((double)ch * (double)ch + (double)sh * (double)sh) - 1.0;
    static constexpr float cl = (float)((double)ch * eps), sl = (float)((double)sh * eps);   // w~ eps
    // k a multiple of N/8: exp(-i pi e8 / 4)
    static constexpr int e8 = (8 * k) % N == 0 ? (8 * k) / N : -1;
};

// x * exp(-i pi e / 4) (FWD) or x * exp(+i pi e / 4) (!FWD): exact swaps and
// sign changes at multiples of pi/2, the split 1/sqrt(2) of dft8 at odd
// multiples of pi/4 (accurate to ~1e-15, so either direction is the other's
// inverse to rounding)
template <int E8, bool FWD> __device__ __forceinline__ float2 rot_eighth(float2 x) {
    constexpr int e = FWD ? (8 - E8) % 8 : E8;   // as a positive rotation
    if constexpr (e == 0) return x;
    else if constexpr (e == 2) return cmul_i(x);
    else if constexpr (e == 4) return make_float2(-x.x, -x.y);
    else if constexpr (e == 6) return cmul_mi(x);
    else if constexpr (e == 1) return make_float2(mul_rsqrt2(x.x - x.y), mul_rsqrt2(x.x + x.y));
    else if constexpr (e == 3) return make_float2(-mul_rsqrt2(x.x + x.y), mul_rsqrt2(x.x - x.y));
    else if constexpr (e == 5) return make_float2(mul_rsqrt2(x.y - x.x), -mul_rsqrt2(x.x + x.y));
    else return make_float2(mul_rsqrt2(x.x + x.y), mul_rsqrt2(x.y - x.x));   // e == 7
}

// forward root: x * w~
template <int K, int N> __device__ __forceinline__ float2 rot_fwd(float2 x) {
    using W = Root<K, N>;
    if constexpr (W::e8 >= 0) return rot_eighth<W::e8, true>(x);
    else return make_float2(fmaf(x.x, W::ch, -x.y * W::sh), fmaf(x.x, W::sh, x.y * W::ch));
}
// its inverse: x * conj(w~ + w~ eps), one rounding per component
template <int K, int N> __device__ __forceinline__ float2 rot_inv(float2 x) {
    using W = Root<K, N>;
    if constexpr (W::e8 >= 0) return rot_eighth<W::e8, false>(x);
    else return cmulconj_hilo(x, make_float2(W::ch, W::sh), make_float2(W::cl, W::sl));
}

// Forward DFT of R = 16 or 32 points in registers, natural order in and out:
// n = n1 + 4 n2, k = k2 + (R/4) k1; inner DFT_{R/4} over n2, roots w_R^(n1 k2),
// outer DFT_4 over n1.
template <int R> __device__ __forceinline__ void dft_4x_fwd(float2 *u) {
    constexpr int Q = R / 4;
    static_for<0, 4>([&](auto n1c) {
        constexpr int n1 = decltype(n1c)::value;
        float2 v[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) v[n2] = u[n1 + 4 * n2];
        dft<Q, -1>(v);
        static_for<0, Q>([&](auto k2c) {
            constexpr int k2 = decltype(k2c)::value;
            u[n1 + 4 * k2] = rot_fwd<n1 * k2, R>(v[k2]);
        });
    });
    float2 o[R];
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
        float2 v[4] = {u[4 * k2], u[4 * k2 + 1], u[4 * k2 + 2], u[4 * k2 + 3]};
        dft4<-1>(v);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) o[k2 + Q * k1] = v[k1];
    }
#pragma unroll
    for (int k = 0; k < R; ++k) u[k] = o[k];
}

// R times the inverse of dft_4x_fwd<R>: its factors in reverse order, each
// inverted (DFT_4 and DFT_{R/4} by their conjugates, the roots by rot_inv).
template <int R> __device__ __forceinline__ void dft_4x_bwd(float2 *u) {
    constexpr int Q = R / 4;
    float2 o[R];
    static_for<0, Q>([&](auto k2c) {
        constexpr int k2 = decltype(k2c)::value;
        float2 v[4] = {u[k2], u[k2 + Q], u[k2 + 2 * Q], u[k2 + 3 * Q]};
        dft4<+1>(v);
        static_for<0, 4>([&](auto n1c) {
            constexpr int n1 = decltype(n1c)::value;
            o[n1 + 4 * k2] = rot_inv<n1 * k2, R>(v[n1]);
        });
    });
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        float2 v[Q];
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k2] = o[n1 + 4 * k2];
        dft<Q, +1>(v);
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) u[n1 + 4 * n2] = v[n2];
    }
}

// DFT_R forward, and R times its inverse (radix 8 and below: dft8's roots are
// the accurate 1/sqrt(2) pair, so the conjugate DFT is the inverse)
template <int R> __device__ __forceinline__ void dft_fwd(float2 *u) {
    if constexpr (R <= 8) dft<R, -1>(u);
    else dft_4x_fwd<R>(u);
}
template <int R> __device__ __forceinline__ void dft_bwd(float2 *u) {
    if constexpr (R <= 8) dft<R, +1>(u);
    else dft_4x_bwd<R>(u);
}

// Stage-2 twiddle entry (c, s, c eps, s eps): c + i s the FP32 rounding of
// w_N^(r j), eps = 1/(c^2 + s^2) - 1.  Forward: x * (c + i s); backward:
// x * conj((c + i s)(1 + eps)), its exact inverse, rounded once.
__device__ __forceinline__ float2 tw_fwd(float2 x, float4 w) {
    return make_float2(fmaf(x.x, w.x, -x.y * w.y), fmaf(x.x, w.y, x.y * w.x));
}
__device__ __forceinline__ float2 tw_bwd(float2 x, float4 w) {
    return cmulconj_hilo(x, make_float2(w.x, w.y), make_float2(w.z, w.w));
}

// Physical row of logical index i during a column exchange: the low three bits
// are XOR-ed with the three bits above log2(E).  With swizzled tile rows (two
// or four columns per warp) both the stage-1 writes and the stage-2 reads then
// spread a column's lanes evenly over the eight 16-byte bank groups.
template <int E> __device__ __forceinline__ int xslot(int i) { return i ^ ((i >> ilog2c(E)) & 7); }

// Twiddle table of the two-stage plan: entry (r - 1) E + j holds w_N^(r j)
// for r in [1, P), j in [0, E) as (c, s, c eps, s eps) (tw_fwd / tw_bwd).
template <int N, int E> __host__ __device__ constexpr int warp_fft_table_size() { return (N / E - 1) * E; }

// The forward transform of the line held by this lane's group of P lanes.
// `xat(i)` is the address of the exchange slot of logical index i (the
// caller's layout spreads both exchange patterns over the banks); the caller
// has synchronised the warp since the slots were last read.  Ends with a
// __syncwarp() before the result is in registers, so the slots may be
// rewritten by the caller.
template <int N, int E, typename XAt, typename Tw>
__device__ __forceinline__ void warp_fft(float2 (&x)[E], int t, const XAt &xat, const Tw &tw) {
    constexpr int P = N / E;
    static_assert(P == 8 || P == 16, "two-stage plan: 8 or 16 lanes per line");
    static_assert(E >= P && E % P == 0, "two-stage plan: E >= P");
    dft_fwd<E>(x);
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
        for (int r = 1; r < P; ++r) u[r] = tw_fwd(x[q + (E / P) * r], tw((r - 1) * E + j));
        dft_fwd<P>(u);
#pragma unroll
        for (int r = 0; r < P; ++r) x[q + (E / P) * r] = u[r];
    }
}

// N times the inverse of warp_fft<N, E>: stage 2 undone (DFT_P inverted, then
// the twiddles), the exchange undone, then DFT_E inverted.  Same
// synchronisation contract as warp_fft.
template <int N, int E, typename XAt, typename Tw>
__device__ __forceinline__ void warp_ifft(float2 (&x)[E], int t, const XAt &xat, const Tw &tw) {
    constexpr int P = N / E;
    static_assert(P == 8 || P == 16, "two-stage plan: 8 or 16 lanes per line");
#pragma unroll
    for (int q = 0; q < E / P; ++q) {
        const int j = t + P * q;
        float2 u[P];
#pragma unroll
        for (int r = 0; r < P; ++r) u[r] = x[q + (E / P) * r];
        dft_bwd<P>(u);
        x[q] = u[0];
#pragma unroll
        for (int r = 1; r < P; ++r) x[q + (E / P) * r] = tw_bwd(u[r], tw((r - 1) * E + j));
    }
#pragma unroll
    for (int m = 0; m < E; ++m) *xat(t + P * m) = x[m];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < E; ++r) x[r] = *xat(E * t + r);
    __syncwarp();
    dft_bwd<E>(x);
}

}  // namespace xsde
