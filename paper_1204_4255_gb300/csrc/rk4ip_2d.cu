// rk4ip_2d.cu -- RK4IP on 2D lattices as four fused passes per step.
//
// XMDS2 (arXiv:1204.4255) Sec. 2.6: exp(L dt/2) is applied by transforming to
// Fourier space, multiplying, and transforming back; Sec. 2.2: the transform of
// a tensor-product lattice factorises per dimension.  Between passes the fields
// are kept transformed along the contiguous dimension 1 only, so
//   row pass    (dimension 1): F1^-1 -> real-space RK4 stage work -> F1
//   column pass (dimension 0): F0 -> * exp(L(k) dt/2)/(n0 n1) -> F0^-1
// and a step is row(S4 of step n-1 + S1 of step n) -> col -> row(S2) -> col.
// Every pass reads two fields and writes two (in place, whole lines per CTA),
// i.e. 16 field accesses per point per step.
#include "fft.cuh"
#include "kernels.h"

namespace xsde {
namespace {

template <int T>
__device__ __forceinline__ void group_sum2(double (&v)[2], int t, double *scratch) {
    // sum over the T threads of a line; T <= 32: xor shuffles inside the group,
    // T > 32: warp sums combined through shared memory (all threads call this)
    if constexpr (T <= 32) {
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < 2; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    } else {
        constexpr int W = T / 32;
        const int line = threadIdx.x / T;
#pragma unroll
        for (int i = 0; i < 2; ++i) v[i] = warp_sum(v[i]);
        __syncthreads();
        if ((t & 31) == 0)
#pragma unroll
            for (int i = 0; i < 2; ++i) scratch[(line * W + (t >> 5)) * 2 + i] = v[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < W; ++w) s += scratch[(line * W + w) * 2 + i];
            v[i] = s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Row pass: T = N1/8 threads per line, LINES lines per CTA.
// ---------------------------------------------------------------------------
template <int N1> struct RowCfg {
    static constexpr int E = 8;
    static constexpr int T = N1 / E;
    static constexpr int LINES = T >= 256 ? 1 : 256 / T;
    static constexpr int THREADS = LINES * T;
};

// TRIG1: dimension 1 is a cosine or sine dimension (p.basis1), see below
template <typename R, int N1, int MODE, bool TRIG1 = false>
__global__ void __launch_bounds__(RowCfg<N1>::THREADS) row_pass_kernel(const Params2D<R> p) {
    using V = cx<R>;
    using Cfg = RowCfg<N1>;
    constexpr int E = Cfg::E, T = Cfg::T, LINES = Cfg::LINES;
    constexpr int BUF = line_len<V, N1>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *smem = reinterpret_cast<V *>(smem_raw);
    const int line = threadIdx.x / T;
    const int t = threadIdx.x - line * T;
    V *const sm2[2] = {smem + line * 2 * BUF, smem + line * 2 * BUF + BUF};
    V *const sm1[1] = {smem + line * 2 * BUF};
    double *scratch = reinterpret_cast<double *>(smem + LINES * 2 * BUF);
    const SyncBlock sync{};
    const TwiddleLdg<tw_t<R>> tw{p.tw1};
    const LineLayout<V> L{};

    const int64_t nrows = p.npaths * (int64_t)p.n0;
    const int64_t row = (int64_t)blockIdx.x * LINES + line;
    // (bounds-checking build: the line's last element inside the field)
    const bool active = row < nrows && XSDE_IN(row * N1 + N1 - 1, nrows * N1, p.status);
    const int64_t rrow = active ? row : 0;
    const int64_t path = rrow / p.n0;
    // line within the path; its lattice indices are (i0) in 2D, (i0, i1) in 3D
    const int i0 = (int)(rrow - path * p.n0);
    const int la = p.ndim == 3 ? i0 / p.nmid : i0;
    const int lb = p.ndim == 3 ? i0 - la * p.nmid : 0;
    const uint32_t gp = (uint32_t)(p.lt.path_offset + path);
    V *Arow = p.A + rrow * N1;
    V *Brow = p.B + rrow * N1;
    const R gdt = p.lt.gdt;
    const R sixth = R(1) / R(6), third = R(1) / R(3), half = R(0.5);
    const bool sample = p.sample_slot >= 0;

    // A cosine / sine dimension 1 (TRIG1; XMDS2 Sec. 2.1) holds a line's points
    // in the even-odd order of the DCT-II's evaluation by an N1-point FFT:
    // register slot s holds point 2s below N1/2 and point 2 N1-1-2s above,
    // negated (with its additive noise) for the sine basis.  Real-space loads
    // and stores gather and scatter through that order; after the forward
    // transform U_k = A_k V_k + B_k V_{N1-k} applies the dimension-1 factor of
    // exp(L dt/2) in that basis (A in E1, B in p.B1; one exchange pairs k with
    // N1-k), where a Fourier line multiplies by E1.
    const int bas1 = TRIG1 ? p.basis1 : 0;
    auto pt_of = [&](int sl) -> int { return !TRIG1 ? sl : (sl < N1 / 2 ? 2 * sl : 2 * N1 - 1 - 2 * sl); };
    auto negated = [&](int sl) -> bool { return TRIG1 && bas1 == 2 && sl >= N1 / 2; };
    auto load_real = [&](const V *f, int sl) -> V {
        const V v = f[pt_of(sl)];
        return negated(sl) ? mk<V>(-v.x, -v.y) : v;
    };
    auto store_real = [&](V *f, int sl, V v) { f[pt_of(sl)] = negated(sl) ? mk<V>(-v.x, -v.y) : v; };

    // raw potential of point (line, t + m T) at global step gs
    auto pot = [&](int m, uint64_t gs) -> R {
        const int ic = pt_of(t + m * T);
        const int idx2[3] = {la, ic, 0};
        const int idx3[3] = {la, lb, ic};
        return potential(p.lt, p.ndim, p.ndim == 3 ? idx3 : idx2, (int64_t)i0 * N1 + ic, gs);
    };
    // static potentials are evaluated once per element; tables with one row per
    // step are read for the step at hand
    const bool vtime = p.lt.pot == PM_TABLE && p.lt.V_nt > 1;
    R Vst[E];
#pragma unroll
    for (int m = 0; m < E; ++m) Vst[m] = vtime ? R(0) : pot(m, 0);
    auto potv = [&](int m, uint64_t gs) -> R { return vtime ? pot(m, gs) : Vst[m]; };
    auto pterm = [&](int m, uint64_t gs) -> PointTerm<R> {
        const int i1 = pt_of(t + m * T);
        PointTerm<R> pt = point_term(p.lt, potv(m, gs), (uint32_t)(i0 * N1 + i1), gp, (uint32_t)gs);
        if (negated(t + m * T)) pt.na = mk<V>(-pt.na.x, -pt.na.y);
        return pt;
    };
    // local part of the sampling group for the real-space field f at global step gs
    // (vnl: the non-local potential of f, whose pair energy 1/2 V_nl |f|^2 the
    // energy adds; nullptr without the term)
    auto sample_local = [&](const V (&f)[E], uint64_t gs, const R *vnl = nullptr) {
        double acc[2] = {0.0, 0.0};
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const double m2 = (double)cabs2(f[m]);
            acc[0] += m2;
            acc[1] += (double)potv(m, gs) * m2 + 0.5 * p.sm.g * m2 * m2;
            if (vnl) acc[1] += 0.5 * (double)vnl[m] * m2;
            if (active && (p.sm.which & (MOM_MOD2 | MOM_MOD4)) && p.sm.per_point) {
                const int64_t ip = (int64_t)p.sample_slot * p.lt.npts + (int64_t)i0 * N1 + pt_of(t + m * T);
                if (!XSDE_IN(ip, p.sm.nsamp * p.lt.npts, p.status)) continue;
                double *pp = p.sm.per_point + 2 * ip;
                atomicAdd(pp, m2 * p.sm.inv_paths);
                atomicAdd(pp + 1, m2 * m2 * p.sm.inv_paths);
            }
        }
        group_sum2<T>(acc, t, scratch);
        if (t == 0 && active) {
            if ((p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path) {
                const int64_t iq = (int64_t)p.sample_slot * p.npaths + path;
                if (!XSDE_IN(iq, p.sm.nsamp * p.npaths, p.status)) return;
                double *pq = p.sm.per_path + 2 * iq;
                atomicAdd(pq, acc[0] * p.sm.dV);
                atomicAdd(pq + 1, acc[1] * p.sm.dV);
            }
            if (!isfinite(acc[0])) atomicOr(p.status, ST_NONFINITE);
        }
    };

    if constexpr (MODE == ROW_SI) {
        // the semi-implicit midpoint step (XMDS2 Sec. 2.5) in the interaction
        // picture on one field; see SiOp for the state between passes
        const int op = p.si_op;
        V y[1][E];
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = Arow[t + m * T];
        auto store_scaled = [&](const V (&f)[E]) {
            if (active)
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const V eh = __ldg(p.E1 + t + m * T), el = __ldg(p.E1 + N1 + t + m * T);
                    Arow[t + m * T] = cmul_hilo(f[m], eh, el);
                }
        };
        if (op == SI_ENTER) {
            fft<N1, E, -1, 1>(y, t, sm1, L, sync, tw);
            const R inv = R(1) / R(N1);
            if (active)
#pragma unroll
                for (int m = 0; m < E; ++m) Arow[t + m * T] = cscale(y[0][m], inv);
            return;
        }
        if (op == SI_MUL) {
            if (sample) {
                V z[1][E];
#pragma unroll
                for (int m = 0; m < E; ++m) z[0][m] = y[0][m];
                fft<N1, E, +1, 1>(z, t, sm1, L, sync, tw);
                sample_local(z[0], p.sg);
            }
            // back to the unnormalised F1 a the column pass expects (a power of two: exact)
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = cscale(y[0][m], R(N1));
            store_scaled(y[0]);
            return;
        }
        fft<N1, E, +1, 1>(y, t, sm1, L, sync, tw);
        if (op == SI_EXIT) {
            if (sample) sample_local(y[0], p.sg);
            if (active)
#pragma unroll
                for (int m = 0; m < E; ++m) Arow[t + m * T] = y[0][m];
            return;
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const PointTerm<R> pt = pterm(m, p.sg);
            V mid = y[0][m];
            for (int it = 0; it < 3; ++it) mid = caxpy(y[0][m], half, apply_N(mid, pt, gdt));
            y[0][m] = mk<V>(R(2) * mid.x - y[0][m].x, R(2) * mid.y - y[0][m].y);
        }
        fft<N1, E, -1, 1>(y, t, sm1, L, sync, tw);
        store_scaled(y[0]);
        return;
    }

    V x[2][E];
    if constexpr (MODE == ROW_NL) {
        // RK4IP with the non-local potential (Example 5) on a 2D lattice: see NlOp
        const int op = p.nl_op;
        V *Crow = p.C + rrow * N1;
        V *Drow = p.D + rrow * N1;
        // C = F1 |u|^2 of this line (the density the column pass convolves)
        auto density_out = [&](const V (&u)[E]) {
            V y[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = mk<V>(cabs2(u[m]), R(0));
            fft<N1, E, -1, 1>(y, t, sm1, L, sync, tw);
            if (active)
#pragma unroll
                for (int m = 0; m < E; ++m) Crow[t + m * T] = y[0][m];
        };
        // V_nl = Re F1^-1 C (C = F1 V_nl after the convolving column pass)
        auto vnl_in = [&](R (&v)[E]) {
            V y[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = Crow[t + m * T];
            fft<N1, E, +1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
            for (int m = 0; m < E; ++m) v[m] = y[0][m].x;
        };
        // the point term of step gs with V_nl added to the potential
        auto ptv = [&](int m, uint64_t gs, R vnl) -> PointTerm<R> {
            PointTerm<R> pt = pterm(m, gs);
            pt.dtV += p.lt.dt * vnl;
            return pt;
        };
        R v[E];
        if (op == NL_DENSITY || op == NL_PROLOGUE || op == NL_FFT) {
#pragma unroll
            for (int m = 0; m < E; ++m) x[0][m] = Arow[t + m * T];
            if (op == NL_DENSITY) {
                density_out(x[0]);
                return;
            }
            vnl_in(v);
            if (sample) sample_local(x[0], p.sg, v);
            if (op == NL_FFT) {
                V y[1][E];
#pragma unroll
                for (int m = 0; m < E; ++m) y[0][m] = x[0][m];
                fft<N1, E, -1, 1>(y, t, sm1, L, sync, tw);
                if (active)
#pragma unroll
                    for (int m = 0; m < E; ++m) Brow[t + m * T] = y[0][m];
                return;
            }
#pragma unroll
            for (int m = 0; m < E; ++m) x[1][m] = apply_N(x[0][m], ptv(m, p.sg, v[m]), gdt);
        } else if (op == NL_SDA) {
            V y[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = Arow[t + m * T];
            fft<N1, E, +1, 1>(y, t, sm1, L, sync, tw);
            density_out(y[0]);
            return;
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                x[0][m] = Arow[t + m * T];
                x[1][m] = Brow[t + m * T];
            }
            fft<N1, E, +1, 2>(x, t, sm2, L, sync, tw);
            if (op == NL_S2A) {
                V u[E];
#pragma unroll
                for (int m = 0; m < E; ++m) u[m] = caxpy(x[0][m], half, x[1][m]);
                density_out(u);
                return;
            }
            vnl_in(v);
            if (op == NL_S2B) {
                V u[E];
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const V k2 = apply_N(caxpy(x[0][m], half, x[1][m]), ptv(m, p.sg, v[m]), gdt);
                    if (active) Drow[t + m * T] = k2;
                    u[m] = caxpy(x[0][m], half, k2);
                }
                density_out(u);
                return;
            }
            if (op == NL_SDB) {
                // k4 = N(D(a_I + k3)) at step sg; a' = D(acc) + k4/6, real space
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    x[0][m] = caxpy(x[1][m], sixth, apply_N(x[0][m], ptv(m, p.sg, v[m]), gdt));
                    if (active) Arow[t + m * T] = x[0][m];
                }
                if (!p.nl_last) density_out(x[0]);
                return;
            }
            // NL_S2C: k3 = N(a_I + k2/2) with the V_nl of that argument
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const V aI = x[0][m], k1 = x[1][m];
                const V k2 = active ? Drow[t + m * T] : mk<V>(R(0), R(0));
                const V k3 = apply_N(caxpy(aI, half, k2), ptv(m, p.sg, v[m]), gdt);
                x[0][m] = cadd(aI, k3);
                x[1][m] = caxpy(caxpy(caxpy(aI, sixth, k1), third, k2), third, k3);
            }
        }
    } else if constexpr (MODE == ROW_PROLOGUE || MODE == ROW_FFT_ONLY) {
#pragma unroll
        for (int m = 0; m < E; ++m) x[0][m] = load_real(Arow, t + m * T);
        if (sample) sample_local(x[0], p.sg);
        if constexpr (MODE == ROW_FFT_ONLY) {
            V y[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) y[0][m] = x[0][m];
            fft<N1, E, -1, 1>(y, t, sm1, L, sync, tw);
            if constexpr (TRIG1) {
                // the cosine spectrum X_k = (w_k V_k + conj(w_k) V_{N1-k}) / 2,
                // w_k = exp(-i pi k / 2 N1) (for the sine basis, mode N1-k at k)
#pragma unroll
                for (int m = 0; m < E; ++m) sm1[0][L(t + m * T)] = y[0][m];
                sync();
                V q[E];
#pragma unroll
                for (int m = 0; m < E; ++m) q[m] = sm1[0][L((N1 - t - m * T) & (N1 - 1))];
                sync();
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    double sn, cs;
                    sincospi(-(double)(t + m * T) / (2.0 * N1), &sn, &cs);
                    const double yr = (double)y[0][m].x, yi = (double)y[0][m].y;
                    const double qr = (double)q[m].x, qi = (double)q[m].y;
                    y[0][m] = mk<V>((R)(0.5 * (cs * (yr + qr) - sn * (yi - qi))),
                                    (R)(0.5 * (cs * (yi + qi) + sn * (yr - qr))));
                }
            }
            if (active)
#pragma unroll
                for (int m = 0; m < E; ++m) Brow[t + m * T] = y[0][m];
            return;
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) x[1][m] = apply_N(x[0][m], pterm(m, p.sg), gdt);
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            x[0][m] = Arow[t + m * T];
            x[1][m] = Brow[t + m * T];
        }
        fft<N1, E, +1, 2>(x, t, sm2, L, sync, tw);
        if constexpr (MODE == ROW_STAGE2) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const PointTerm<R> pt = pterm(m, p.sg);
                const V aI = x[0][m], k1 = x[1][m];
                const V k2 = apply_N(caxpy(aI, half, k1), pt, gdt);
                const V k3 = apply_N(caxpy(aI, half, k2), pt, gdt);
                x[0][m] = cadd(aI, k3);
                x[1][m] = caxpy(caxpy(caxpy(aI, sixth, k1), third, k2), third, k3);
            }
        } else {
            // k4 = N(D(a_I + k3)) at step sg; a' = D(acc) + k4/6
#pragma unroll
            for (int m = 0; m < E; ++m) x[0][m] = caxpy(x[1][m], sixth, apply_N(x[0][m], pterm(m, p.sg), gdt));
            if constexpr (MODE == ROW_EPILOGUE) {
                if (active)
#pragma unroll
                    for (int m = 0; m < E; ++m) store_real(Arow, t + m * T, x[0][m]);
                return;
            } else {
                if (sample) sample_local(x[0], p.sg + 1);
#pragma unroll
                for (int m = 0; m < E; ++m) x[1][m] = apply_N(x[0][m], pterm(m, p.sg + 1), gdt);
            }
        }
    }
    fft<N1, E, -1, 2>(x, t, sm2, L, sync, tw);
    // the dimension-1 factor of exp(L dt/2); the column pass applies the rest
    if constexpr (TRIG1) {
        V q[2][E];
#pragma unroll
        for (int m = 0; m < E; ++m)
#pragma unroll
            for (int iv = 0; iv < 2; ++iv) sm2[iv][L(t + m * T)] = x[iv][m];
        sync();
#pragma unroll
        for (int m = 0; m < E; ++m)
#pragma unroll
            for (int iv = 0; iv < 2; ++iv) q[iv][m] = sm2[iv][L((N1 - t - m * T) & (N1 - 1))];
        sync();
        if (active)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int j = t + m * T;
                const V ah = __ldg(p.E1 + j), al = __ldg(p.E1 + N1 + j);
                const V bh = __ldg(p.B1 + j), bl = __ldg(p.B1 + N1 + j);
                Arow[j] = cadd(cmul_hilo(x[0][m], ah, al), cmul_hilo(q[0][m], bh, bl));
                Brow[j] = cadd(cmul_hilo(x[1][m], ah, al), cmul_hilo(q[1][m], bh, bl));
            }
    } else if (active) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const V eh = __ldg(p.E1 + t + m * T), el = __ldg(p.E1 + N1 + t + m * T);
            Arow[t + m * T] = cmul_hilo(x[0][m], eh, el);
            Brow[t + m * T] = cmul_hilo(x[1][m], eh, el);
        }
    }
}

// ---------------------------------------------------------------------------
// Column pass: a tile of C adjacent columns of one path; T = N0/E threads per
// column; lanes run over columns first so every load is a 128-byte segment.
// ---------------------------------------------------------------------------
template <typename R, int N0> struct ColCfg {
    // 128-byte row segments (16 c64 / 8 c128 columns) up to 1024 (c64) or 512
    // (c128) threads per CTA; longer columns use narrower tiles.
    static constexpr int CMAX = sizeof(R) == 4 ? 16 : 8;
    static constexpr int TMAX = sizeof(R) == 4 ? 1024 : 512;
    static constexpr int E = 8;
    static constexpr int T = N0 / E;
    static constexpr int C0 = (CMAX * T <= TMAX) ? CMAX : TMAX / T;
    // at least one full warp per CTA (the sample reductions use whole-warp shuffles)
    static constexpr int C = (C0 * T < 32) ? 32 / T : C0;
    static constexpr int THREADS = C * T;
    static_assert(THREADS % 32 == 0, "column tiles are whole warps");
};

template <typename R, int N0, int MODE, bool TRIG = false>
__global__ void __launch_bounds__(ColCfg<R, N0>::THREADS) col_pass_kernel(const Params2D<R> p) {
    using V = cx<R>;
    using Cfg = ColCfg<R, N0>;
    constexpr int C = Cfg::C, E = Cfg::E, T = Cfg::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *smem = reinterpret_cast<V *>(smem_raw);
    V *const sm2[2] = {smem, smem + N0 * C};
    V *const sm1[1] = {smem};
    double *scratch = reinterpret_cast<double *>(smem + 2 * N0 * C);
    const int c = threadIdx.x % C;
    const int t = threadIdx.x / C;
    const SyncBlock sync{};
    const TwiddleLdg<tw_t<R>> tw{p.tw0};
    const ColumnTile<C> L{c};

    const int col = blockIdx.x * C + c;
    const int64_t path = blockIdx.y;
    const int n1 = p.n1;
    const int64_t base = path * (int64_t)N0 * n1 + col;
    const bool sample = p.sample_slot >= 0;
#if XSDE_BOUNDS
    // the column's last element inside the field (one decision for the CTA)
    if (!__syncthreads_and(XSDE_IN(base + (int64_t)(N0 - 1) * n1, p.npaths * (int64_t)N0 * n1, p.status) &&
                           XSDE_IN(col, n1, p.status)))
        return;
#endif
    // A cosine / sine dimension 0 (TRIG; XMDS2 Sec. 2.1) gathers its rows in the
    // even-odd order of the DCT-II's evaluation by an N0-point FFT (slot s holds
    // row 2s below N0/2, row 2 N0-1-2s above; odd rows negated for the sine
    // basis); between the FFTs one exchange pairs k with N0-k and
    // U_k = A_k V_k + B_k V_{N0-k} applies exp(L dt/2) in the cosine / sine basis.
    const int bas = TRIG ? p.basis0 : 0;
    auto row_of = [&](int s) -> int { return !TRIG ? s : (s < N0 / 2 ? 2 * s : 2 * N0 - 1 - 2 * s); };
    auto at = [&](int s) -> int64_t { return base + (int64_t)row_of(s) * n1; };
    auto load = [&](const V *f, int s) -> V {
        const V v = f[at(s)];
        return (TRIG && bas == 2 && s >= N0 / 2) ? mk<V>(-v.x, -v.y) : v;
    };
    auto store = [&](V *f, int s, V v) { f[at(s)] = (TRIG && bas == 2 && s >= N0 / 2) ? mk<V>(-v.x, -v.y) : v; };
    // partner values V_{N0-k} of the transformed vectors (TRIG)
    auto partners = [&](auto &v, auto &q) {
        constexpr int NV = sizeof(v) / sizeof(v[0]);
#pragma unroll
        for (int m = 0; m < E; ++m)
#pragma unroll
            for (int iv = 0; iv < NV; ++iv) sm2[iv][L(t + m * T)] = v[iv][m];
        sync();
#pragma unroll
        for (int m = 0; m < E; ++m)
#pragma unroll
            for (int iv = 0; iv < NV; ++iv) q[iv][m] = sm2[iv][L((N0 - t - m * T) & (N0 - 1))];
        sync();
    };

    auto kinetic = [&](const V (&f)[E], const V (&fq)[E]) {
        // sum_k Re(i L(k)) |F psi|^2 dV / N, accumulated into the energy of this path.
        // The column index is k1 (2D) or the pair (k1, k2) = (col / kinner, col % kinner) (3D).
        double kc2;
        double wc = 1.0;   // Parseval weights of cosine / sine dimensions 1 and 2
        if (p.kinner > 0) {
            const int ia = col / p.kinner, ib = col - ia * p.kinner, nm = n1 / p.kinner;
            // a cosine / sine dimension holds its cosine spectrum (sine mode n-k
            // at k), weight 2 for every mode but slot 0
            const double ka = p.sm.kscale[1] * (p.basis1 == 1 ? ia : p.basis1 == 2 ? nm - ia
                                                                   : (ia < nm / 2 ? ia : ia - nm));
            const double kb = p.sm.kscale[2] * (p.basis2 == 1 ? ib : p.basis2 == 2 ? p.kinner - ib
                                                                   : (ib < p.kinner / 2 ? ib : ib - p.kinner));
            if (p.basis1 && ia != 0) wc *= 2.0;
            if (p.basis2 && ib != 0) wc *= 2.0;
            kc2 = ka * ka + kb * kb;
        } else if (p.basis1) {
            // cosine / sine dimension 1: B holds the cosine spectrum X_k1 (sine
            // mode n1-k1 at k1); Parseval weight 2 for every mode but slot 0
            const double k1 = p.sm.kscale[1] * (p.basis1 == 1 ? col : n1 - col);
            kc2 = k1 * k1;
        } else {
            const double k1 = p.sm.kscale[1] * (col < n1 / 2 ? col : col - n1);
            kc2 = k1 * k1;
        }
        // fields written by propagating row passes already carry the
        // dimension-1 factor of exp(L dt/2); divide its modulus back out
        const double w = (MODE == COL_SPECTRAL) ? p.spec_scale : 1.0 / (double)cabs2(p.E1[col]);
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int kj = t + m * T;
            if constexpr (TRIG) {
                // cosine spectrum from the pair, Parseval weight 2 but at k = 0;
                // sine mode N0-1-k sits at k
                double sn, cs;
                sincospi(-(double)kj / (2.0 * N0), &sn, &cs);
                const double xr = 0.5 * (cs * ((double)f[m].x + (double)fq[m].x) - sn * ((double)f[m].y - (double)fq[m].y));
                const double xi = 0.5 * (cs * ((double)f[m].y + (double)fq[m].y) + sn * ((double)f[m].x - (double)fq[m].x));
                const double k0 = p.sm.kscale[0] * (bas == 1 ? kj : N0 - kj);
                s += (kj == 0 ? 1.0 : 2.0) * (p.sm.h0 + p.sm.h2 * (k0 * k0 + kc2)) * (xr * xr + xi * xi);
            } else {
                const double k0 = p.sm.kscale[0] * (kj < N0 / 2 ? kj : kj - N0);
                s += (p.sm.h0 + p.sm.h2 * (k0 * k0 + kc2)) * (double)cabs2(f[m]);
            }
        }
        if (p.basis1 && p.kinner == 0 && col != 0) wc = 2.0;
        s *= w * wc;
        s = warp_sum(s);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += scratch[w];
            if ((p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path)
                if (XSDE_IN((int64_t)p.sample_slot * p.npaths + path, p.sm.nsamp * p.npaths, p.status))
                atomicAdd(p.sm.per_path + 2 * ((int64_t)p.sample_slot * p.npaths + path) + 1,
                          tot * p.sm.dV / ((double)N0 * n1));
        }
    };

    if constexpr (MODE == COL_CONV) {
        // C <- F0^-1 K2(k0, col) F0 C: the density convolution of the non-local
        // term (the kernel of a pair function is not separable per dimension)
        V y[1][E];
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = p.C[base + (int64_t)(t + m * T) * n1];
        fft<N0, E, -1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = cmul(y[0][m], __ldg(p.K2 + (int64_t)(t + m * T) * n1 + col));
        fft<N0, E, +1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) p.C[base + (int64_t)(t + m * T) * n1] = y[0][m];
        return;
    } else if constexpr (MODE == COL_SINGLE) {
        V y[1][E];
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = load(p.A, t + m * T);
        fft<N0, E, -1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const V eh = __ldg(p.E0 + t + m * T), el = __ldg(p.E0 + N0 + t + m * T);
            y[0][m] = cmul_hilo(y[0][m], eh, el);
        }
        fft<N0, E, +1, 1>(y, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) store(p.A, t + m * T, y[0][m]);
        return;
    } else if constexpr (MODE == COL_SPECTRAL || MODE == COL_FFT_FWD || MODE == COL_FFT_BWD) {
        V y[1][E];
#pragma unroll
        for (int m = 0; m < E; ++m) y[0][m] = load(p.B, t + m * T);
        fft<N0, E, MODE == COL_FFT_BWD ? +1 : -1, 1>(y, t, sm1, L, sync, tw);
        if constexpr (MODE == COL_SPECTRAL) {
            V yq[1][E];
            if constexpr (TRIG) partners(y, yq);
            kinetic(y[0], yq[0]);
        } else {
            if constexpr (TRIG && MODE == COL_FFT_FWD) {
                // a cosine / sine dimension 1 of a 3D sample: the cosine spectrum
                // X_k = (w_k V_k + conj(w_k) V_{N0-k}) / 2, w_k = exp(-i pi k / 2 N0)
                V yq[1][E];
                partners(y, yq);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    double sn, cs;
                    sincospi(-(double)(t + m * T) / (2.0 * N0), &sn, &cs);
                    const double yr = (double)y[0][m].x, yi = (double)y[0][m].y;
                    const double qr = (double)yq[0][m].x, qi = (double)yq[0][m].y;
                    y[0][m] = mk<V>((R)(0.5 * (cs * (yr + qr) - sn * (yi - qi))),
                                    (R)(0.5 * (cs * (yi + qi) + sn * (yr - qr))));
                }
            }
#pragma unroll
            for (int m = 0; m < E; ++m) p.B[base + (int64_t)(t + m * T) * n1] = y[0][m];   // 3D only
        }
        return;
    } else {
        V x[2][E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            x[0][m] = load(p.A, t + m * T);
            x[1][m] = load(p.B, t + m * T);
        }
        fft<N0, E, -1, 2>(x, t, sm2, L, sync, tw);
        V xq[2][E];
        if constexpr (TRIG) partners(x, xq);
        if (sample) kinetic(x[0], xq[0]);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const V eh = __ldg(p.E0 + t + m * T), el = __ldg(p.E0 + N0 + t + m * T);
            if constexpr (TRIG) {
                const V bh = __ldg(p.B0 + t + m * T), bl = __ldg(p.B0 + N0 + t + m * T);
                x[0][m] = cadd(cmul_hilo(x[0][m], eh, el), cmul_hilo(xq[0][m], bh, bl));
                x[1][m] = cadd(cmul_hilo(x[1][m], eh, el), cmul_hilo(xq[1][m], bh, bl));
            } else {
                x[0][m] = cmul_hilo(x[0][m], eh, el);
                x[1][m] = cmul_hilo(x[1][m], eh, el);
            }
        }
        fft<N0, E, +1, 2>(x, t, sm2, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            store(p.A, t + m * T, x[0][m]);
            store(p.B, t + m * T, x[1][m]);
        }
    }
}

template <typename R, int N1, int MODE> cudaError_t row_launch(const Params2D<R> &p, cudaStream_t s) {
    using Cfg = RowCfg<N1>;
    const size_t smem = (size_t)Cfg::LINES * 2 * line_len<cx<R>, N1>() * sizeof(cx<R>) +
                        (size_t)Cfg::LINES * (Cfg::T / 32 + 1) * 2 * sizeof(double);
    auto kern = row_pass_kernel<R, N1, MODE>;
    if constexpr (MODE == ROW_PROLOGUE || MODE == ROW_STAGE2 || MODE == ROW_STEADY || MODE == ROW_EPILOGUE ||
                  MODE == ROW_FFT_ONLY) {
        if (p.basis1) kern = row_pass_kernel<R, N1, MODE, true>;
    } else if (p.basis1) {
        return cudaErrorInvalidValue;   // the semi-implicit and non-local modes: Fourier lines only
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = p.npaths * (int64_t)p.n0;
    const int64_t blocks = (rows + Cfg::LINES - 1) / Cfg::LINES;
    kern<<<(unsigned)blocks, Cfg::THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, int N1> cudaError_t row_mode(int mode, const Params2D<R> &p, cudaStream_t s) {
    switch (mode) {
        case ROW_PROLOGUE: return row_launch<R, N1, ROW_PROLOGUE>(p, s);
        case ROW_STAGE2: return row_launch<R, N1, ROW_STAGE2>(p, s);
        case ROW_STEADY: return row_launch<R, N1, ROW_STEADY>(p, s);
        case ROW_EPILOGUE: return row_launch<R, N1, ROW_EPILOGUE>(p, s);
        case ROW_FFT_ONLY: return row_launch<R, N1, ROW_FFT_ONLY>(p, s);
        case ROW_SI: return row_launch<R, N1, ROW_SI>(p, s);
        case ROW_NL: return row_launch<R, N1, ROW_NL>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R, int N0, int MODE> cudaError_t col_launch(const Params2D<R> &p, cudaStream_t s) {
    using Cfg = ColCfg<R, N0>;
    const size_t smem = (size_t)2 * N0 * Cfg::C * sizeof(cx<R>) + (Cfg::THREADS / 32 + 1) * sizeof(double);
    auto kern = col_pass_kernel<R, N0, MODE>;
    if constexpr (MODE != COL_FFT_BWD && MODE != COL_SINGLE && MODE != COL_CONV)
        if (p.basis0) kern = col_pass_kernel<R, N0, MODE, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(p.n1 / Cfg::C), (unsigned)p.npaths);
    kern<<<grid, Cfg::THREADS, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, int N0> cudaError_t col_mode(int mode, const Params2D<R> &p, cudaStream_t s) {
    if (p.n1 % ColCfg<R, N0>::C) return cudaErrorInvalidValue;
    switch (mode) {
        case COL_PROPAGATE: return col_launch<R, N0, COL_PROPAGATE>(p, s);
        case COL_SPECTRAL: return col_launch<R, N0, COL_SPECTRAL>(p, s);
        case COL_FFT_FWD: return col_launch<R, N0, COL_FFT_FWD>(p, s);
        case COL_SINGLE: return col_launch<R, N0, COL_SINGLE>(p, s);
        case COL_CONV: return col_launch<R, N0, COL_CONV>(p, s);
        case COL_FFT_BWD: return col_launch<R, N0, COL_FFT_BWD>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace


template <typename R> cudaError_t launch_row_pass(int mode, const Params2D<R> &p, cudaStream_t s) {
    switch (p.n1) {
        case 16: return row_mode<R, 16>(mode, p, s);
        case 32: return row_mode<R, 32>(mode, p, s);
        case 64: return row_mode<R, 64>(mode, p, s);
        case 128: return row_mode<R, 128>(mode, p, s);
        case 256: return row_mode<R, 256>(mode, p, s);
        case 512: return row_mode<R, 512>(mode, p, s);
        case 1024: return row_mode<R, 1024>(mode, p, s);
        case 2048: return row_mode<R, 2048>(mode, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename R> cudaError_t launch_col_pass(int mode, const Params2D<R> &p, cudaStream_t s) {
    if (p.basis0 && (mode == COL_FFT_BWD || mode == COL_SINGLE || mode == COL_CONV)) return cudaErrorInvalidValue;
    switch (p.n0) {
        case 16: return col_mode<R, 16>(mode, p, s);
        case 32: return col_mode<R, 32>(mode, p, s);
        case 64: return col_mode<R, 64>(mode, p, s);
        case 128: return col_mode<R, 128>(mode, p, s);
        case 256: return col_mode<R, 256>(mode, p, s);
        case 512: return col_mode<R, 512>(mode, p, s);
        case 1024: return col_mode<R, 1024>(mode, p, s);
        case 2048: return col_mode<R, 2048>(mode, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// XSDE_REAL_BITS selects one precision and XSDE_PART the row (0) or column (1)
// passes per translation unit (parallel builds)
#if !defined(XSDE_PART) || XSDE_PART == 0
#define XSDE_2D_ROW(R) template cudaError_t launch_row_pass<R>(int, const Params2D<R> &, cudaStream_t);
#else
#define XSDE_2D_ROW(R)
#endif
#if !defined(XSDE_PART) || XSDE_PART == 1
#define XSDE_2D_COL(R) template cudaError_t launch_col_pass<R>(int, const Params2D<R> &, cudaStream_t);
#else
#define XSDE_2D_COL(R)
#endif
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 32
XSDE_2D_ROW(float)
XSDE_2D_COL(float)
#endif
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 64
XSDE_2D_ROW(double)
XSDE_2D_COL(double)
#endif

}  // namespace xsde
