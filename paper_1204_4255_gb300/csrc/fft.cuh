// fft.cuh -- register-distributed Stockham FFTs for the RK4IP kernels.
//
// A length-N transform is carried by T = N/E threads.  Thread t holds the E
// elements x[t + m*T], m = 0..E-1, in registers, both on entry and on exit (the
// Stockham autosort keeps natural order).  Stages have radix R in {2, 4, 8}
// (the first stage takes the remainder of log2 N, the others the largest radix
// that divides E), each thread doing E/R butterflies per stage; between stages
// the values cross threads through a shared-memory buffer whose index map is
// supplied by the caller (padded rows, or column tiles).  The last stage ends
// in registers, so a transform costs (stages - 1) shared-memory exchanges.
//
// Stage with radix R after Ns = product of earlier radices (Ns*R <= N):
//   butterfly j in [0, N/R): inputs x[j + r*N/R]; k = j mod Ns;
//   u_r = x[j + r*N/R] * w^(r*k) with w = exp(S 2 pi i / (Ns R));
//   U = DFT_R(u) with sign S;  y[(j - k) R + k + r Ns] = U_r.
// Forward transforms (S = -1) are unnormalised; inverse ones (S = +1) are the
// plain sum with conjugate roots (callers fold 1/N into other factors).
// This is the spectral-to-spatial transform of XMDS2 Sec. 2.2 for the Fourier
// basis of Sec. 2.1, written for sm_103a register files and shared memory.
#pragma once

#include "device_common.cuh"

namespace xsde {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// radix of the stage that starts when `rem` points remain to be combined
template <int E> __host__ __device__ constexpr int stage_radix(int rem) {
    constexpr int rmax = E >= 8 ? 8 : E;
    constexpr int lr = ilog2c(rmax);
    return (ilog2c(rem) % lr) ? (1 << (ilog2c(rem) % lr)) : rmax;
}

// Twiddles are stored per stage: the stage starting at Ns with radix R holds
// w_N^(r k N/(Ns R)) at [offset(Ns) + (r-1) Ns + k], r in [1,R), k in [0,Ns),
// so the lanes of a warp (consecutive k) read consecutive entries.  The radix
// plan depends on E only through the largest radix min(E, 8): one table serves
// every E >= 8, others need the table of their own plan.
template <int E> __host__ __device__ constexpr int stage_table_offset(int N, int Ns) {
    int off = 0, ns = 1;
    while (ns < Ns) {
        const int R = stage_radix<E>(N / ns);
        if (ns > 1) off += (R - 1) * ns;
        ns *= R;
    }
    return off;
}
__host__ __device__ constexpr int stage_table_offset(int N, int Ns) { return stage_table_offset<8>(N, Ns); }
__host__ __device__ constexpr int stage_table_size(int N) { return stage_table_offset(N, N); }

// ---------------------------------------------------------------------------
// small DFTs in registers, natural-order output
// ---------------------------------------------------------------------------
template <int S, typename V> __device__ __forceinline__ void dft2(V *u) {
    V a = u[0];
    u[0] = cadd(a, u[1]);
    u[1] = csub(a, u[1]);
}

template <int S, typename V> __device__ __forceinline__ void dft4(V *u) {
    V s02 = cadd(u[0], u[2]), d02 = csub(u[0], u[2]);
    V s13 = cadd(u[1], u[3]), d13 = csub(u[1], u[3]);
    V r = (S < 0) ? cmul_mi(d13) : cmul_i(d13);    // S*i*(u1 - u3)
    u[0] = cadd(s02, s13);
    u[2] = csub(s02, s13);
    u[1] = cadd(d02, r);
    u[3] = csub(d02, r);
}

// a / sqrt(2).  In FP32 the constant is split hi + lo and applied with one FMA:
// the rounded constant alone has 2 h^2 = 1 - 3.4e-8, a bias that every radix-8
// stage would add to the norm of the field (thousands of stages per run).
__device__ __forceinline__ float mul_rsqrt2(float a) { return fmaf(0.70710677f, a, 1.21016175e-08f * a); }
__device__ __forceinline__ double mul_rsqrt2(double a) { return 0.70710678118654752440084436210485 * a; }

template <int S, typename V> __device__ __forceinline__ void dft8(V *u) {
    V e[4] = {u[0], u[2], u[4], u[6]};
    V o[4] = {u[1], u[3], u[5], u[7]};
    dft4<S>(e);
    dft4<S>(o);
    // o[k] *= exp(S 2 pi i k / 8)
    if (S < 0) {
        o[1] = mk<V>(mul_rsqrt2(o[1].x + o[1].y), mul_rsqrt2(o[1].y - o[1].x));
        o[2] = cmul_mi(o[2]);
        o[3] = mk<V>(mul_rsqrt2(o[3].y - o[3].x), -mul_rsqrt2(o[3].x + o[3].y));
    } else {
        o[1] = mk<V>(mul_rsqrt2(o[1].x - o[1].y), mul_rsqrt2(o[1].x + o[1].y));
        o[2] = cmul_i(o[2]);
        o[3] = mk<V>(-mul_rsqrt2(o[3].x + o[3].y), mul_rsqrt2(o[3].x - o[3].y));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        u[k] = cadd(e[k], o[k]);
        u[k + 4] = csub(e[k], o[k]);
    }
}

template <int R, int S, typename V> __device__ __forceinline__ void dft(V *u) {
    if constexpr (R == 2) dft2<S>(u);
    else if constexpr (R == 4) dft4<S>(u);
    else dft8<S>(u);
}

// ---------------------------------------------------------------------------
// Twiddles.  FP64: (cos, sin).  FP32: (cos_hi, sin_hi, cos_lo, sin_lo), the
// FP64 value split into a rounded pair and its rounded remainder, applied by
// cmul_hilo so every twiddle acts with ~46-bit accuracy.  (FP32 twiddles alone
// sit ~1e-8 below unit modulus on average at the angles the early stages use;
// a butterfly with a unit-modulus twiddle is unitary, one without it drains
// ~1e-8 of the norm per transform, i.e. ~1e-4 over a 2000-step 2D run.)
// ---------------------------------------------------------------------------
template <typename R> struct tw_of;
template <> struct tw_of<float> { using type = float4; };
template <> struct tw_of<double> { using type = double2; };
template <typename R> using tw_t = typename tw_of<R>::type;

// u * w (S < 0) or u * conj(w) (S > 0)
template <int S> __device__ __forceinline__ float2 twiddle_mul(float2 u, float4 w) {
    const float2 hi = make_float2(w.x, w.y), lo = make_float2(w.z, w.w);
    return (S < 0) ? cmul_hilo(u, hi, lo) : cmulconj_hilo(u, hi, lo);
}
template <int S> __device__ __forceinline__ double2 twiddle_mul(double2 u, double2 w) {
    return (S < 0) ? cmul(u, w) : cmulconj(u, w);
}

// ---------------------------------------------------------------------------
// one stage on NV vectors held by this thread
// ---------------------------------------------------------------------------
template <int N, int E, int R, int Ns, int S, int NV, typename V, typename Tw>
__device__ __forceinline__ void fft_stage(V (&v)[NV][E], int t, const Tw &tw) {
    constexpr int B = E / R, T = N / E;
    using TW = decltype(tw(0));
#pragma unroll
    for (int q = 0; q < B; ++q) {
        TW w[R];
        if constexpr (Ns > 1) {
            const int k = (t + q * T) & (Ns - 1);
            constexpr int off = stage_table_offset<E>(N, Ns);
#pragma unroll
            for (int r = 1; r < R; ++r) w[r] = tw(off + (r - 1) * Ns + k);
        }
#pragma unroll
        for (int iv = 0; iv < NV; ++iv) {
            V u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[iv][q + r * B];
            if constexpr (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) u[r] = twiddle_mul<S>(u[r], w[r]);
            }
            dft<R, S>(u);
#pragma unroll
            for (int r = 0; r < R; ++r) v[iv][q + r * B] = u[r];
        }
    }
}

// Move stage outputs to their Stockham positions and fetch the next inputs.
// sm[iv] is the exchange buffer of vector iv; L maps logical index -> slot.
template <typename Layout> struct odd_swap_first {
    static constexpr bool value = false;
};

template <int N, int E, int R, int Ns, int NV, typename V, typename Layout, typename Sync>
__device__ __forceinline__ void fft_exchange(V (&v)[NV][E], int t, V *const (&sm)[NV], const Layout &L,
                                             const Sync &sync) {
    constexpr int B = E / R, T = N / E;
    // In the first exchange, threads t and t+1 write lines R apart.  Layouts
    // where that lands both in the same banks have odd t write its R outputs in
    // pairwise-swapped order, so simultaneous writes are R +- 1 lines apart.
    constexpr bool swap = Ns == 1 && odd_swap_first<Layout>::value;
    const bool odd = swap && (t & 1);
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = t + q * T;
        const int k = j & (Ns - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if constexpr (swap) {
                const int slot = L(base + (odd ? (r ^ 1) : r));
#pragma unroll
                for (int iv = 0; iv < NV; ++iv) sm[iv][slot] = odd ? v[iv][q + (r ^ 1) * B] : v[iv][q + r * B];
            } else {
                const int slot = L(base + r * Ns);
#pragma unroll
                for (int iv = 0; iv < NV; ++iv) sm[iv][slot] = v[iv][q + r * B];
            }
        }
    }
    sync();
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int slot = L(t + m * T);
#pragma unroll
        for (int iv = 0; iv < NV; ++iv) v[iv][m] = sm[iv][slot];
    }
    sync();
}

template <int N, int E, int S, int Ns, int NV, typename V, typename Layout, typename Sync, typename Tw>
__device__ __forceinline__ void fft_from(V (&v)[NV][E], int t, V *const (&sm)[NV], const Layout &L,
                                         const Sync &sync, const Tw &tw) {
    constexpr int R = stage_radix<E>(N / Ns);
    static_assert(E % R == 0, "radix must divide the elements per thread");
    fft_stage<N, E, R, Ns, S, NV>(v, t, tw);
    if constexpr (Ns * R < N) {
        fft_exchange<N, E, R, Ns, NV>(v, t, sm, L, sync);
        fft_from<N, E, S, Ns * R, NV>(v, t, sm, L, sync, tw);
    }
}

// Transform NV vectors in lockstep (sign S; see the header comment).
template <int N, int E, int S, int NV, typename V, typename Layout, typename Sync, typename Tw>
__device__ __forceinline__ void fft(V (&v)[NV][E], int t, V *const (&sm)[NV], const Layout &L,
                                    const Sync &sync, const Tw &tw) {
    static_assert((N & (N - 1)) == 0 && N >= E, "N must be a power of two, at least E");
    static_assert(N % E == 0, "E must divide N");
    fft_from<N, E, S, 1, NV>(v, t, sm, L, sync, tw);
}

// --- paired complex64 transforms ---------------------------------------------
// fftp_fwd is fft<N, E, -1> with every twiddle applied as its FP32 rounding
// w~ alone; fftp_bwd is N times its exact inverse: the stages and exchanges
// undone in reverse order, each butterfly by the conjugate DFT_R (dft8's
// 1/sqrt(2) is accurate to ~1e-15) and each twiddle by 1/w~ = conj(w~)(1 + eps),
// eps = 1/|w~|^2 - 1, applied from the pair (w~, w~ eps) with one rounding per
// component.  Table entries (c, s, c eps, s eps) in the per-stage layout.  A
// forward / backward pair is the identity up to rounding whatever the modulus
// of the rounded twiddles, which is what keeps a long run's norm: plain FP32
// twiddles in both directions drain ~1e-4 over 2000 2D steps.
__device__ __forceinline__ float2 twp_fwd(float2 x, float4 w) {
    return make_float2(fmaf(x.x, w.x, -x.y * w.y), fmaf(x.x, w.y, x.y * w.x));
}
__device__ __forceinline__ float2 twp_bwd(float2 x, float4 w) {
    return cmulconj_hilo(x, make_float2(w.x, w.y), make_float2(w.z, w.w));
}

// Paired twiddles staged in shared memory as two float2 arrays, (c, s) and
// (c eps, s eps): the forward transform reads only the first, 8 bytes a lane
// at an 8-byte stride (a float4 entry read for its first half would put lanes
// 8 entries apart on the same banks).  The row pass uses it (its shared-memory
// pipe is ~60 % busy); the warp column pass keeps float4 entries, where two
// 8-byte reads per backward twiddle cost more issue than they save.
struct PairedTwiddles {
    const float2 *hi, *lo;
    __device__ __forceinline__ float4 operator()(int m) const {
        const float2 h = hi[m], l = lo[m];
        return make_float4(h.x, h.y, l.x, l.y);
    }
};
// stage a paired table of n float4 entries from global memory into hi / lo
__device__ __forceinline__ void stage_paired(float2 *hi, float2 *lo, const float4 *g, int n, int tid, int nthreads) {
    for (int i = tid; i < n; i += nthreads) {
        const float4 w = g[i];
        hi[i] = make_float2(w.x, w.y);
        lo[i] = make_float2(w.z, w.w);
    }
}

template <int N, int E, int R, int Ns, bool FWD, int NV, typename Tw>
__device__ __forceinline__ void fftp_stage(float2 (&v)[NV][E], int t, const Tw &tw) {
    constexpr int B = E / R, T = N / E;
#pragma unroll
    for (int q = 0; q < B; ++q) {
        float4 w[R];
        if constexpr (Ns > 1) {
            const int k = (t + q * T) & (Ns - 1);
            constexpr int off = stage_table_offset<E>(N, Ns);
#pragma unroll
            for (int r = 1; r < R; ++r) w[r] = tw(off + (r - 1) * Ns + k);
        }
#pragma unroll
        for (int iv = 0; iv < NV; ++iv) {
            float2 u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[iv][q + r * B];
            if constexpr (FWD) {
                if constexpr (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < R; ++r) u[r] = twp_fwd(u[r], w[r]);
                }
                dft<R, -1>(u);
            } else {
                dft<R, +1>(u);
                if constexpr (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < R; ++r) u[r] = twp_bwd(u[r], w[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) v[iv][q + r * B] = u[r];
        }
    }
}

// the inverse permutation of fft_exchange<N, E, R, Ns>
template <int N, int E, int R, int Ns, int NV, typename V, typename Layout, typename Sync>
__device__ __forceinline__ void fft_exchange_back(V (&v)[NV][E], int t, V *const (&sm)[NV], const Layout &L,
                                                  const Sync &sync) {
    constexpr int B = E / R, T = N / E;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int slot = L(t + m * T);
#pragma unroll
        for (int iv = 0; iv < NV; ++iv) sm[iv][slot] = v[iv][m];
    }
    sync();
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = t + q * T;
        const int k = j & (Ns - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int slot = L(base + r * Ns);
#pragma unroll
            for (int iv = 0; iv < NV; ++iv) v[iv][q + r * B] = sm[iv][slot];
        }
    }
    sync();
}

template <int N, int E, int Ns, int NV, typename Layout, typename Sync, typename Tw>
__device__ __forceinline__ void fftp_fwd_from(float2 (&v)[NV][E], int t, float2 *const (&sm)[NV], const Layout &L,
                                              const Sync &sync, const Tw &tw) {
    constexpr int R = stage_radix<E>(N / Ns);
    static_assert(E % R == 0, "radix must divide the elements per thread");
    fftp_stage<N, E, R, Ns, true, NV>(v, t, tw);
    if constexpr (Ns * R < N) {
        fft_exchange<N, E, R, Ns, NV>(v, t, sm, L, sync);
        fftp_fwd_from<N, E, Ns * R, NV>(v, t, sm, L, sync, tw);
    }
}
template <int N, int E, int Ns, int NV, typename Layout, typename Sync, typename Tw>
__device__ __forceinline__ void fftp_bwd_from(float2 (&v)[NV][E], int t, float2 *const (&sm)[NV], const Layout &L,
                                              const Sync &sync, const Tw &tw) {
    constexpr int R = stage_radix<E>(N / Ns);
    if constexpr (Ns * R < N) {
        fftp_bwd_from<N, E, Ns * R, NV>(v, t, sm, L, sync, tw);
        fft_exchange_back<N, E, R, Ns, NV>(v, t, sm, L, sync);
    }
    fftp_stage<N, E, R, Ns, false, NV>(v, t, tw);
}
template <int N, int E, int NV, typename Layout, typename Sync, typename Tw>
__device__ __forceinline__ void fftp_fwd(float2 (&v)[NV][E], int t, float2 *const (&sm)[NV], const Layout &L,
                                         const Sync &sync, const Tw &tw) {
    fftp_fwd_from<N, E, 1, NV>(v, t, sm, L, sync, tw);
}
template <int N, int E, int NV, typename Layout, typename Sync, typename Tw>
__device__ __forceinline__ void fftp_bwd(float2 (&v)[NV][E], int t, float2 *const (&sm)[NV], const Layout &L,
                                         const Sync &sync, const Tw &tw) {
    fftp_bwd_from<N, E, 1, NV>(v, t, sm, L, sync, tw);
}

// --- index maps and barriers ------------------------------------------------

// Exchange buffer of one line.  8-byte elements (complex64): rows of 16 slots
// (128 bytes) whose low four index bits are XOR-ed with (5 x row) mod 16; a
// wavefront count of every exchange of the radix-2/4/8 plans (16..2048 points,
// 8/4/2 elements per thread) puts it within 0.2 % of conflict-free, where one
// pad slot every 8 was 48 % above.  A slot stays in its row, so the buffer
// holds N slots.  16-byte elements (complex128): one pad slot every 8, already
// conflict-free for these patterns.
template <typename V> struct LineLayout {
    __device__ __forceinline__ int operator()(int i) const {
        if constexpr (sizeof(V) == 8) return i ^ (((i >> 4) * 5) & 15);
        else return i + (i >> 3);
    }
};
template <typename V, int N> __host__ __device__ constexpr int line_len() { return sizeof(V) == 8 ? N : N + N / 8; }

// tile of C lines interleaved element by element (slot = i*C + c)
template <int C> struct ColumnTile {
    int c;
    __device__ __forceinline__ int operator()(int i) const { return i * C + c; }
};
// 8 complex64 columns: a row is 64 B, so two rows an even distance apart share
// banks, and a half-warp (two threads per column) writing lines R apart conflicts
template <> struct odd_swap_first<ColumnTile<8>> {
    static constexpr bool value = true;
};

struct SyncBlock {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncWarp {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
// named barrier `id` shared by `count` threads (count a multiple of 32)
struct SyncNamed {
    int id, count;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
    }
};

// twiddles exp(-2 pi i m / N) from a table
template <typename V> struct TwiddleTable {
    const V *p;
    __device__ __forceinline__ V operator()(int m) const { return p[m]; }
};
template <typename V> struct TwiddleLdg {
    const V *p;
    __device__ __forceinline__ V operator()(int m) const { return __ldg(p + m); }
};

}  // namespace xsde
