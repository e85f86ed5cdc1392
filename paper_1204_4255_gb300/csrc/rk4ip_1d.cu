// rk4ip_1d.cu -- whole-run RK4IP for 1D lattices (N <= 2048), one CTA slot per path.
//
// XMDS2 (arXiv:1204.4255) Sec. 2.5 (method of lines, RK4) with Sec. 2.6 (the
// interaction picture, re-centred each step so only exp(L dt/2) is needed).
// Per step, with D(u) = F^-1 exp(L dt/2) F u and N(u) = dt g(u):
//   a_I = D a,  k1 = D N(a),  k2 = N(a_I + k1/2),  k3 = N(a_I + k2/2),
//   k4 = N(D(a_I + k3)),  a <- D(a_I + k1/6 + k2/3 + k3/3) + k4/6.
// The field never leaves the SM during the run: each thread keeps the points
// t + m*T (m < 8) of its path in registers, the eight FFTs of a step exchange
// through shared memory, and D is applied to two vectors in lockstep.  Only the
// initial load, the final store, time-dependent potential rows and the FP64
// samples touch global memory.
#include "fft.cuh"
#include "kernels.h"

namespace xsde {
namespace {

// barrier of the T threads that carry one path
template <int T, int PPC> struct SlotSync {
    int slot;
    __device__ __forceinline__ void operator()() const {
        if constexpr (T <= 32) __syncwarp();
        else if constexpr (PPC == 1) __syncthreads();
        else asm volatile("bar.sync %0, %1;" ::"r"(slot + 1), "r"(T) : "memory");
    }
};

// sum three doubles over the T threads of a slot (result in every thread)
template <int T, typename Sync>
__device__ __forceinline__ void slot_sum3(double (&v)[3], int t, double *scratch, const Sync &sync) {
    if constexpr (T <= 32) {
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    } else {
        constexpr int W = T / 32;
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = warp_sum(v[i]);
        sync();
        if ((t & 31) == 0)
#pragma unroll
            for (int i = 0; i < 3; ++i) scratch[(t >> 5) * 3 + i] = v[i];
        sync();
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) s += scratch[w * 3 + i];
            v[i] = s;
        }
        sync();
    }
}

// the step's point term with the non-local potential vn added to V
template <typename R> __device__ __forceinline__ PointTerm<R> with_vnl(PointTerm<R> pt, R dt, R vn) {
    pt.dtV += dt * vn;
    return pt;
}

// NOISE: the problem has Wiener noise (a template flag, so deterministic runs
// carry no generator code)
// NL: g carries the non-local potential V_nl = Re F^-1[khat F|psi|^2] of
// XMDS2 Example 5 (Sec. 3.5): every evaluation of N transforms the density of
// its argument forward and back once more (one vector, same exchange buffer)
// SCHEME 1: the semi-implicit midpoint step in the interaction picture instead
// of RK4IP (a_I = D a; m <- a_I + N(m)/2 three times from m = a_I;
// a <- D(2 m - a_I): XMDS2 Sec. 2.5's semi-implicit method with Sec. 2.6)
// TRIG: a cosine or sine lattice (XMDS2 Sec. 2.1; p.basis 1 / 2), see below
// MINB: CTAs per SM the register allocation must allow (1: no cap)
template <typename R, int N, int E, int PPC, bool NOISE, int SCHEME = 0, bool NL = false, bool TRIG = false,
          int MINB = 1>
__global__ void __launch_bounds__(PPC *(N / E), MINB) rk4ip_1d_kernel(const Params1D<R> p) {
    using V = cx<R>;
    constexpr int T = N / E;
    constexpr int BUF = line_len<V, N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tw_t<R> *tws = reinterpret_cast<tw_t<R> *>(smem_raw);
    const int slot = threadIdx.x / T;
    const int t = threadIdx.x - slot * T;
    V *bufA = reinterpret_cast<V *>(tws + N) + slot * 2 * BUF;
    V *bufB = bufA + BUF;
    V *const sm2[2] = {bufA, bufB};
    V *const sm1[1] = {bufA};
    const SlotSync<T, PPC> sync{slot};
    const TwiddleTable<tw_t<R>> tw{tws};
    const LineLayout<V> L{};

    for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = p.tw[i];
    __syncthreads();

    // Cosine / sine lattices (TRIG).  The N cell-centred points are held in
    // the even-odd order of the DCT-II's evaluation by an N-point FFT
    // (Makhoul, IEEE TASSP 1980): register slot s holds point 2s for s < N/2
    // and point 2N-1-2s above.  The FFT of the slots, V, gives the cosine
    // spectrum X_k = (w_k V_k + conj(w_k) V_{N-k})/2, w_k = exp(-i pi k/2N), and
    // D = C^-1 diag(E) C becomes U_k = A_k V_k + B_k V_{N-k} between the two
    // FFTs (A, B from the host; one exchange pairs k with N-k).  A sine
    // lattice is the cosine one of (-1)^j psi_j with its modes reversed: its
    // odd points (slots s >= N/2) are held negated, and so is their additive
    // noise.  Real-space work at slot s uses point point_of(s).
    const int bas = TRIG ? p.basis : 0;
    auto point_of = [&](int s) -> int { return !TRIG ? s : (s < N / 2 ? 2 * s : 2 * N - 1 - 2 * s); };
    auto negated = [&](int s) -> bool { return TRIG && bas == 2 && s >= N / 2; };
    const int64_t lp = (int64_t)blockIdx.x * PPC + slot;
    const bool active = lp < p.npaths;
    const uint32_t gp = (uint32_t)(p.lt.path_offset + lp);
    V *psi = p.psi + lp * N;
    const bool vtime = p.lt.pot == PM_TABLE && p.lt.V_nt > 1;

    V x[2][E];
    V Ek[E], El[E];   // exp(L dt/2)/N (Fourier) or A (TRIG), hi and lo; B is read through L1
    R Vs[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + m * T;
        const int pj = point_of(j);
        x[0][m] = (active && XSDE_IN(lp * N + pj, p.npaths * N, p.status)) ? psi[pj] : mk<V>(R(0), R(0));
        if (negated(j)) x[0][m] = mk<V>(-x[0][m].x, -x[0][m].y);
        Ek[m] = p.Etab[j];
        El[m] = p.Etab[N + j];
        const int idx[3] = {pj, 0, 0};
        Vs[m] = vtime ? R(0) : potential(p.lt, 1, idx, pj, 0);
    }

    // exp(L dt/2) in the lattice's spectral basis, on NV transformed vectors
    auto kmul = [&](auto &v) {
        constexpr int NV = sizeof(v) / sizeof(v[0]);
        if constexpr (TRIG) {
            V *const *smv = NV == 2 ? sm2 : sm1;
#pragma unroll
            for (int m = 0; m < E; ++m)
#pragma unroll
                for (int iv = 0; iv < NV; ++iv) smv[iv][L(t + m * T)] = v[iv][m];
            sync();
            V q[NV][E];
#pragma unroll
            for (int m = 0; m < E; ++m)
#pragma unroll
                for (int iv = 0; iv < NV; ++iv) q[iv][m] = smv[iv][L((N - t - m * T) & (N - 1))];
            sync();
#pragma unroll
            for (int m = 0; m < E; ++m)
#pragma unroll
                for (int iv = 0; iv < NV; ++iv)
                    v[iv][m] = cadd(cmul_hilo(v[iv][m], Ek[m], El[m]),
                                    cmul_hilo(q[iv][m], __ldg(p.Btab + t + m * T), __ldg(p.Btab + N + t + m * T)));
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m)
#pragma unroll
                for (int iv = 0; iv < NV; ++iv) v[iv][m] = cmul_hilo(v[iv][m], Ek[m], El[m]);
        }
    };
    const R gdt = p.lt.gdt;
    const R sixth = R(1) / R(6), third = R(1) / R(3), half = R(0.5);

    // vn = V_nl of the slot's field u (khat is stored divided by N, so both
    // transforms stay unnormalised)
    auto nonlocal = [&](const V (&u)[E], R (&vn)[E]) {
        V y[1][E];
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = mk<V>(cabs2(u[m]), R(0));
        fft<N, E, -1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = cmul(y[0][m], p.knl[t + m * T]);
        fft<N, E, +1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) vn[m] = y[0][m].x;
    };
    R vn[E];

    for (int64_t n = 0;; ++n) {
        // ---- sampling group (XMDS2 Sec. 2.5 moments over paths) ----------
        if (p.sm.every > 0 && n % p.sm.every == 0) {
            const int64_t s = n / p.sm.every;
            const uint64_t gs = p.step0 + n;
            double acc[3] = {0.0, 0.0, 0.0};   // norm, local energy, kinetic energy
            if constexpr (NL) nonlocal(x[0], vn);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int j = point_of(t + m * T);
                const int idx[3] = {j, 0, 0};
                const double m2 = (double)cabs2(x[0][m]);
                const double vv = (double)potential(p.lt, 1, idx, j, gs);
                acc[0] += m2;
                acc[1] += vv * m2 + 0.5 * p.sm.g * m2 * m2;
                if constexpr (NL) acc[1] += 0.5 * (double)vn[m] * m2;   // pair energy, counted once
                if (active && (p.sm.which & (MOM_MOD2 | MOM_MOD4)) && p.sm.per_point &&
                    XSDE_IN(s * N + j, p.sm.nsamp * N, p.status)) {
                    double *pp = p.sm.per_point + 2 * (s * N + j);
                    atomicAdd(pp, m2 * p.sm.inv_paths);
                    atomicAdd(pp + 1, m2 * m2 * p.sm.inv_paths);
                }
            }
            V y[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = x[0][m];
            fft<N, E, -1, 1>(y, t, sm1, L, sync, tw);
            if constexpr (TRIG) {
                // cosine spectrum X_k from the pair (k, N-k); Parseval weight 2
                // for every mode but k = 0; sine mode N-1-k sits at k
#pragma unroll
                for (int m = 0; m < E; ++m) bufA[L(t + m * T)] = y[0][m];
                sync();
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int kj = t + m * T;
                    const V yq = bufA[L((N - kj) & (N - 1))];
                    double sn, cs;
                    sincospi(-(double)kj / (2.0 * N), &sn, &cs);
                    const double xr = 0.5 * (cs * ((double)y[0][m].x + (double)yq.x) - sn * ((double)y[0][m].y - (double)yq.y));
                    const double xi = 0.5 * (cs * ((double)y[0][m].y + (double)yq.y) + sn * ((double)y[0][m].x - (double)yq.x));
                    const double k = p.sm.kscale[0] * (bas == 1 ? kj : N - kj);
                    acc[2] += (kj == 0 ? 1.0 : 2.0) * (p.sm.h0 + p.sm.h2 * k * k) * (xr * xr + xi * xi);
                }
                sync();
            } else {
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const int kj = t + m * T;
                    const double k = p.sm.kscale[0] * (kj < N / 2 ? kj : kj - N);
                    acc[2] += (p.sm.h0 + p.sm.h2 * k * k) * (double)cabs2(y[0][m]);
                }
            }
            slot_sum3<T>(acc, t, reinterpret_cast<double *>(bufB), sync);
            if (t == 0 && active) {
                const double norm = acc[0] * p.sm.dV;
                if ((p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path &&
                    XSDE_IN(s * p.npaths + lp, p.sm.nsamp * p.npaths, p.status)) {
                    double *pq = p.sm.per_path + 2 * (s * p.npaths + lp);
                    pq[0] = norm;
                    pq[1] = (acc[1] + acc[2] / N) * p.sm.dV;
                }
                if (!isfinite(norm)) atomicOr(p.status, ST_NONFINITE);
            }
        }
        if (n == p.nsteps) break;

        // ---- one RK4IP step ----------------------------------------------
        const uint64_t sg = p.step0 + n;
        PointTerm<R> pt[E];
        if constexpr (NL) nonlocal(x[0], vn);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + m * T;
            const int pj = point_of(j);
            R v = Vs[m];
            if (vtime) v = XSDE_IN((int64_t)sg * N + pj, p.lt.V_nt * N, p.status) ? p.lt.V[(int64_t)sg * N + pj] : R(0);
            if constexpr (NOISE) {
                pt[m] = point_term(p.lt, v, (uint32_t)pj, gp, (uint32_t)sg);
                if (negated(j)) pt[m].na = mk<V>(-pt[m].na.x, -pt[m].na.y);
            } else {
                pt[m].dtV = p.lt.dt * v;
                pt[m].na = mk<V>(R(0), R(0));
            }
            x[1][m] = apply_N(x[0][m], NL ? with_vnl(pt[m], p.lt.dt, vn[m]) : pt[m], gdt);     // N(a)
        }
        if constexpr (SCHEME == 1) {
            V y[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = x[0][m];
            fft<N, E, -1, 1>(y, t, sm1, L, sync, tw);
            kmul(y);
            fft<N, E, +1, 1>(y, t, sm1, L, sync, tw);       // a_I
#pragma unroll
            for (int m = 0; m < E; ++m) {
                V mid = y[0][m];
                for (int it = 0; it < 3; ++it) mid = caxpy(y[0][m], half, apply_N(mid, pt[m], gdt));
                y[0][m] = mk<V>(R(2) * mid.x - y[0][m].x, R(2) * mid.y - y[0][m].y);
            }
            fft<N, E, -1, 1>(y, t, sm1, L, sync, tw);
            kmul(y);
            fft<N, E, +1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
            for (int m = 0; m < E; ++m) x[0][m] = y[0][m];
        } else {
            // a_I = D a and k1 = D N(a) (h = 0), then the k2/k3 stage and
            // D(a_I + k3), D(acc) (h = 1).  The half-step loop stays rolled so the
            // step's code holds one copy of the two-vector transforms (the
            // instruction cache keeps the whole step).
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                if (h == 1) {
                    // k2, k3 in real space; x[0] <- a_I + k3, x[1] <- a_I + k1/6 + k2/3 + k3/3
                    if constexpr (NL) {
                        // V_nl of each stage input needs the whole line: two passes over m
                        V w[E];
#pragma unroll
                        for (int m = 0; m < E; ++m) w[m] = caxpy(x[0][m], half, x[1][m]);
                        nonlocal(w, vn);
#pragma unroll
                        for (int m = 0; m < E; ++m) {
                            const V k2 = apply_N(w[m], with_vnl(pt[m], p.lt.dt, vn[m]), gdt);
                            x[1][m] = caxpy(caxpy(x[0][m], sixth, x[1][m]), third, k2);
                            w[m] = caxpy(x[0][m], half, k2);
                        }
                        nonlocal(w, vn);
#pragma unroll
                        for (int m = 0; m < E; ++m) {
                            const V k3 = apply_N(w[m], with_vnl(pt[m], p.lt.dt, vn[m]), gdt);
                            x[1][m] = caxpy(x[1][m], third, k3);
                            x[0][m] = cadd(x[0][m], k3);
                        }
                    } else {
#pragma unroll
                        for (int m = 0; m < E; ++m) {
                            const V aI = x[0][m], k1 = x[1][m];
                            const V k2 = apply_N(caxpy(aI, half, k1), pt[m], gdt);
                            const V k3 = apply_N(caxpy(aI, half, k2), pt[m], gdt);
                            x[0][m] = cadd(aI, k3);
                            x[1][m] = caxpy(caxpy(caxpy(aI, sixth, k1), third, k2), third, k3);
                        }
                    }
                }
                fft<N, E, -1, 2>(x, t, sm2, L, sync, tw);
                kmul(x);
                fft<N, E, +1, 2>(x, t, sm2, L, sync, tw);
            }
            // k4 = N(D(a_I + k3)); a <- D(acc) + k4/6
            if constexpr (NL) nonlocal(x[0], vn);
#pragma unroll
            for (int m = 0; m < E; ++m)
                x[0][m] = caxpy(x[1][m], sixth, apply_N(x[0][m], NL ? with_vnl(pt[m], p.lt.dt, vn[m]) : pt[m], gdt));
        }
    }

    if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + m * T;
            if (XSDE_IN(lp * N + point_of(j), p.npaths * N, p.status))
                psi[point_of(j)] = negated(j) ? mk<V>(-x[0][m].x, -x[0][m].y) : x[0][m];
        }
    }
}

template <typename R, int N, int E, int PPC, int SCHEME = 0, bool NL = false, bool TRIG = false, int MINB = 1>
cudaError_t launch_ppc(const Params1D<R> &p, cudaStream_t s) {
    constexpr int T = N / E;
    const size_t smem = (size_t)N * sizeof(tw_t<R>) + (size_t)PPC * 2 * line_len<cx<R>, N>() * sizeof(cx<R>);
    const bool noise = p.lt.noise != NM_NONE;
    auto kern = noise ? rk4ip_1d_kernel<R, N, E, PPC, true, SCHEME, NL, TRIG, MINB>
                      : rk4ip_1d_kernel<R, N, E, PPC, false, SCHEME, NL, TRIG, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = (p.npaths + PPC - 1) / PPC;
    kern<<<(unsigned)blocks, PPC * T, smem, s>>>(p);
    return cudaGetLastError();
}

// default paths per CTA for E elements per thread: fill 128 threads
template <int N, int E> constexpr int default_ppc() { return N / E >= 128 ? 1 : 128 / (N / E); }

}  // namespace

// Launch shapes.  Variants 0-3 keep 8 elements per thread (radix-8 stages):
// the default paths per CTA, a half, a quarter (at least one; more CTAs for
// small ensembles) and twice as many (at most 256 threads, so no variant is
// squeezed below 255 registers a thread).  Variants 4 and 5 spread a path over
// more threads, 4 or 2 elements each (radix-4 or radix-2 stages): more warps
// per path for few, long, latency-bound paths.
template <typename R, int N> cudaError_t launch_1d_n(int variant, const Params1D<R> &p, cudaStream_t s) {
    constexpr int P0 = default_ppc<N, 8>(), T = N / 8;
    constexpr int P1 = P0 >= 2 ? P0 / 2 : 1, P2 = P0 >= 4 ? P0 / 4 : 1;
    constexpr int P3 = 2 * P0 * T <= 256 ? 2 * P0 : P0;
    if (p.basis)   // one launch shape for cosine / sine lattices,
        return p.scheme == 1 ? launch_ppc<R, N, 8, P0, 1, false, true>(p, s) : launch_ppc<R, N, 8, P0, 0, false, true>(p, s);
    // 512 resident threads per SM cap a thread at 128 registers: the complex64
    // transforms gain more from the extra warps than they lose to the few
    // spilled values; complex128 keeps all its registers.  Variant 6 takes
    // the other choice.
    constexpr int CAP = P0 * T < 512 ? 512 / (P0 * T) : 1;
    constexpr int MB0 = sizeof(R) == 4 ? CAP : 1, MB6 = sizeof(R) == 4 ? 1 : CAP;
    if (p.scheme == 1) return launch_ppc<R, N, 8, P0, 1, false, false, MB0>(p, s);   // for the semi-implicit step
    if (p.knl) return launch_ppc<R, N, 8, P0, 0, true>(p, s);       // and for the non-local term
    switch (variant) {
        case 1: return launch_ppc<R, N, 8, P1>(p, s);
        case 2: return launch_ppc<R, N, 8, P2>(p, s);
        case 3: return launch_ppc<R, N, 8, P3>(p, s);
        case 4: return launch_ppc<R, N, 4, default_ppc<N, 4>()>(p, s);
        case 5: return launch_ppc<R, N, 2, default_ppc<N, 2>()>(p, s);
        case 6: return launch_ppc<R, N, 8, P0, 0, false, false, MB6>(p, s);
        default: return launch_ppc<R, N, 8, P0, 0, false, false, MB0>(p, s);
    }
}

template <typename R> cudaError_t launch_rk4ip_1d(int n, int variant, const Params1D<R> &p, cudaStream_t s) {
    switch (n) {
        case 16: return launch_1d_n<R, 16>(variant, p, s);
        case 32: return launch_1d_n<R, 32>(variant, p, s);
        case 64: return launch_1d_n<R, 64>(variant, p, s);
        case 128: return launch_1d_n<R, 128>(variant, p, s);
        case 256: return launch_1d_n<R, 256>(variant, p, s);
        case 512: return launch_1d_n<R, 512>(variant, p, s);
        case 1024: return launch_1d_n<R, 1024>(variant, p, s);
        case 2048: return launch_1d_n<R, 2048>(variant, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// Parallel builds: XSDE_REAL_BITS selects one precision and XSDE_PART (0..7)
// one length, 16 << XSDE_PART, per translation unit; part 0 also holds the
// dispatch, which sees the other lengths as extern instantiations.
#define XSDE_1D_N(X, R, N) X template cudaError_t launch_1d_n<R, N>(int, const Params1D<R> &, cudaStream_t);
#if !defined(XSDE_PART) || XSDE_PART == 0
#define XSDE_1D_P0(R) XSDE_1D_N(, R, 16)
#elif XSDE_PART == 0
#define XSDE_1D_P0(R) XSDE_1D_N(extern, R, 16)
#else
#define XSDE_1D_P0(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 1
#define XSDE_1D_P1(R) XSDE_1D_N(, R, 32)
#elif XSDE_PART == 0
#define XSDE_1D_P1(R) XSDE_1D_N(extern, R, 32)
#else
#define XSDE_1D_P1(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 2
#define XSDE_1D_P2(R) XSDE_1D_N(, R, 64)
#elif XSDE_PART == 0
#define XSDE_1D_P2(R) XSDE_1D_N(extern, R, 64)
#else
#define XSDE_1D_P2(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 3
#define XSDE_1D_P3(R) XSDE_1D_N(, R, 128)
#elif XSDE_PART == 0
#define XSDE_1D_P3(R) XSDE_1D_N(extern, R, 128)
#else
#define XSDE_1D_P3(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 4
#define XSDE_1D_P4(R) XSDE_1D_N(, R, 256)
#elif XSDE_PART == 0
#define XSDE_1D_P4(R) XSDE_1D_N(extern, R, 256)
#else
#define XSDE_1D_P4(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 5
#define XSDE_1D_P5(R) XSDE_1D_N(, R, 512)
#elif XSDE_PART == 0
#define XSDE_1D_P5(R) XSDE_1D_N(extern, R, 512)
#else
#define XSDE_1D_P5(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 6
#define XSDE_1D_P6(R) XSDE_1D_N(, R, 1024)
#elif XSDE_PART == 0
#define XSDE_1D_P6(R) XSDE_1D_N(extern, R, 1024)
#else
#define XSDE_1D_P6(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 7
#define XSDE_1D_P7(R) XSDE_1D_N(, R, 2048)
#elif XSDE_PART == 0
#define XSDE_1D_P7(R) XSDE_1D_N(extern, R, 2048)
#else
#define XSDE_1D_P7(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 0
#define XSDE_1D_DISPATCH(R) template cudaError_t launch_rk4ip_1d<R>(int, int, const Params1D<R> &, cudaStream_t);
#else
#define XSDE_1D_DISPATCH(R)
#endif
#define XSDE_1D_UNIT(R)                                                                       \
    XSDE_1D_P0(R) XSDE_1D_P1(R) XSDE_1D_P2(R) XSDE_1D_P3(R) XSDE_1D_P4(R) XSDE_1D_P5(R) XSDE_1D_P6(R) \
    XSDE_1D_P7(R) XSDE_1D_DISPATCH(R)

#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 32
#if !defined(XSDE_PART) || XSDE_PART == 0
int rk4ip_1d_variants() { return 7; }
int rk4ip_1d_elems(int variant) { return variant == 4 ? 4 : variant == 5 ? 2 : 8; }
#endif
XSDE_1D_UNIT(float)
#endif
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 64
XSDE_1D_UNIT(double)
#endif

}  // namespace xsde
