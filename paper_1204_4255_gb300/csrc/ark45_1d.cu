// ark45_1d.cu -- adaptive Cash-Karp 4(5) Runge-Kutta on 1D lattices, in the
// interaction picture or on the explicit equation.
//
// XMDS2 (arXiv:1204.4255) Sec. 2.5 lists an adaptive fourth-fifth order
// Runge-Kutta (Cash & Karp 1990) for deterministic problems, and Sec. 2.6 runs
// it in the interaction picture; Fig. IPvsEX compares the steps it needs with
// and without the picture.  Deterministic equation df/dt = L f + g(f),
// g(f) = -i (V(x) + g |f|^2) f.  One step of size h from t:
//   interaction picture: k_i = h exp(-L c_i h) g(exp(L c_i h) Y_i),
//     Y_i = f + sum_j a_ij k_j, f5 = f + sum_i b5_i k_i, then f <- exp(L h) f5
//     (the picture is re-centred at every step);
//   explicit: k_i = h (L Y_i + g(Y_i)), f <- f + sum_i b5_i k_i.
// Error e = sum_i (b5_i - b4_i) k_i, err = max_j |e_j| / max_j |f5_j| (FP64 block
// reduction); accept if err <= tol; next h = h clamp(0.9 (tol/err)^(1/5),
// 0.2, 5) (5 if err = 0); a step that would pass t_end, or end within 1e-12
// t_end of it, ends on t_end.  tol <= 0: fixed steps of h0.
//
// One CTA per path (its own step size and decisions, uniform over the CTA);
// each thread holds the points t + m*T of the state and of the running sums
// f5 and e in registers, the six stage derivatives live in a global workspace
// that only the owning thread reads back (no synchronisation), and every
// transform runs through shared memory as in rk4ip_1d.cu.  The propagator
// factors exp(L(k) tau) are evaluated per step and node in FP64.
#include "fft.cuh"
#include "kernels.h"

namespace xsde {
namespace {

// Cash & Karp (1990), ACM TOMS 16, 201
__constant__ double kC[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
__constant__ double kA[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
__constant__ double kB5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
__constant__ double kB4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0,
                              1.0 / 4.0};

__device__ __forceinline__ double block_max(double v, double *red, int t, int T) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < T / 32; ++w) m = fmax(m, red[w]);
    return m;
}

// exp(z) / n for z = (c0 + c2 k^2) tau, and exp(-z) / n, in FP64
struct Factor {
    double2 fwd, bwd;
};
__device__ __forceinline__ Factor prop_factor(const double c0r, const double c0i, const double c2r,
                                              const double c2i, double k2, double tau, double inv_n) {
    const double zr = (c0r + c2r * k2) * tau, zi = (c0i + c2i * k2) * tau;
    double s, c;
    sincos(zi, &s, &c);
    const double ep = exp(zr) * inv_n, em = exp(-zr) * inv_n;
    return {make_double2(ep * c, ep * s), make_double2(em * c, -em * s)};
}

template <typename V> __device__ __forceinline__ V cmul_d(V u, double2 f) {
    using R = decltype(V::x);
    const R fx = (R)f.x, fy = (R)f.y;
    return mk<V>(u.x * fx - u.y * fy, u.x * fy + u.y * fx);
}

template <typename R, int N, int E>
__global__ void __launch_bounds__(N / E) ark45_1d_kernel(const AdaptiveParams<R> p) {
    using V = cx<R>;
    constexpr int T = N / E;
    constexpr int BUF = line_len<V, N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tw_t<R> *tws = reinterpret_cast<tw_t<R> *>(smem_raw);
    V *buf = reinterpret_cast<V *>(tws + N);
    double *red = reinterpret_cast<double *>(buf + BUF);   // 64 doubles
    V *const sm1[1] = {buf};
    const SyncBlock sync{};
    const TwiddleTable<tw_t<R>> tw{tws};
    const LineLayout<V> L{};
    const int t = threadIdx.x;
    const int64_t path = blockIdx.x;
    if (!XSDE_IN(path, p.npaths, p.status)) return;   // whole CTA: one path each

    for (int i = t; i < N; i += T) tws[i] = p.tw[i];
    __syncthreads();

    V *psi = p.psi + path * N;
    V *K = p.kbuf + path * 6 * N;
    V y[E];
    R Vs[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + m * T;
        y[m] = psi[j];
        const int idx[3] = {j, 0, 0};
        Vs[m] = potential(p.lt, 1, idx, j, 0);
    }
    // |k|^2 of the frequency element m holds after a forward transform
    auto k2_of = [&](int m) -> double {
        const int j = t + m * T;
        const double k = p.kscale * (j < N / 2 ? j : j - N);
        return k * k;
    };
    const R gnl = (R)p.gnl;
    auto g_of = [&](V u, int m) -> V {   // g(u) = -i (V + g |u|^2) u
        const R s = Vs[m] + gnl * cabs2(u);
        return mk<V>(s * u.y, -s * u.x);
    };
    const double inv_n = 1.0 / N;
    // x <- exp(+-L tau) x: transform, multiply, transform back
    auto propagate = [&](V (&x)[1][E], double tau, bool back) {
        fft<N, E, -1, 1>(x, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const Factor f = prop_factor(p.c0_re, p.c0_im, p.c2_re, p.c2_im, k2_of(m), tau, inv_n);
            x[0][m] = cmul_d(x[0][m], back ? f.bwd : f.fwd);
        }
        fft<N, E, +1, 1>(x, t, sm1, L, sync, tw);
    };

    double tn = 0.0, h = p.h0;
    int64_t acc = 0, rej = 0;
    int st = 0;
    while (tn < p.t_end) {
        if (acc + rej >= p.max_steps) {
            st = ST_STEP_LIMIT;
            break;
        }
        if (tn + h > p.t_end || p.t_end - (tn + h) <= 1e-12 * p.t_end) h = p.t_end - tn;
        V y5[E], er[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            y5[m] = y[m];
            er[m] = mk<V>(R(0), R(0));
        }
        for (int i = 0; i < 6; ++i) {
            V x[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                V s = y[m];
                for (int jj = 0; jj < i; ++jj) {
                    const V kj = K[jj * N + t + m * T];
                    const R a = (R)kA[i][jj];
                    s = mk<V>(s.x + a * kj.x, s.y + a * kj.y);
                }
                x[0][m] = s;
            }
            if (p.picture) {
                const double tau = kC[i] * h;
                if (i > 0) propagate(x, tau, false);
#pragma unroll
                for (int m = 0; m < E; ++m) x[0][m] = g_of(x[0][m], m);
                if (i > 0) propagate(x, tau, true);
#pragma unroll
                for (int m = 0; m < E; ++m) x[0][m] = cscale(x[0][m], (R)h);
            } else {
                V gy[E];
#pragma unroll
                for (int m = 0; m < E; ++m) gy[m] = g_of(x[0][m], m);
                fft<N, E, -1, 1>(x, t, sm1, L, sync, tw);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const double k2 = k2_of(m);
                    const double2 l = make_double2((p.c0_re + p.c2_re * k2) * inv_n, (p.c0_im + p.c2_im * k2) * inv_n);
                    x[0][m] = cmul_d(x[0][m], l);
                }
                fft<N, E, +1, 1>(x, t, sm1, L, sync, tw);
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const V s = mk<V>(x[0][m].x + gy[m].x, x[0][m].y + gy[m].y);
                    x[0][m] = cscale(s, (R)h);
                }
            }
            const R b5 = (R)kB5[i], de = (R)(kB5[i] - kB4[i]);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                if (i < 5) K[i * N + t + m * T] = x[0][m];
                y5[m] = mk<V>(y5[m].x + b5 * x[0][m].x, y5[m].y + b5 * x[0][m].y);
                er[m] = mk<V>(er[m].x + de * x[0][m].x, er[m].y + de * x[0][m].y);
            }
        }
        double emax = 0.0, ymax = 0.0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            emax = fmax(emax, hypot((double)er[m].x, (double)er[m].y));
            ymax = fmax(ymax, hypot((double)y5[m].x, (double)y5[m].y));
        }
        emax = block_max(emax, red, t, T);
        ymax = block_max(ymax, red + 32, t, T);
        const double err = ymax > 0.0 ? emax / ymax : 0.0;
        if (!(err == err)) {   // NaN: the field is no longer finite
            st = ST_NONFINITE;
            break;
        }
        if (p.tol <= 0.0 || err <= p.tol) {
            tn += h;
            ++acc;
            if (p.picture) {
                V x[1][E];
#pragma unroll
                for (int m = 0; m < E; ++m) x[0][m] = y5[m];
                propagate(x, h, false);
#pragma unroll
                for (int m = 0; m < E; ++m) y[m] = x[0][m];
            } else {
#pragma unroll
                for (int m = 0; m < E; ++m) y[m] = y5[m];
            }
        } else {
            ++rej;
        }
        if (p.tol > 0.0) {
            double fac = err > 0.0 ? 0.9 * pow(p.tol / err, 0.2) : 5.0;
            fac = fac < 0.2 ? 0.2 : (fac > 5.0 ? 5.0 : fac);
            h *= fac;
        } else {
            h = p.h0;
        }
    }
#pragma unroll
    for (int m = 0; m < E; ++m) psi[t + m * T] = y[m];
    if (t == 0) {
        p.accepted[path] = acc;
        p.rejected[path] = rej;
        if (st) atomicOr(p.status, st);
    }
}

template <typename R, int N> cudaError_t ark_launch(const AdaptiveParams<R> &p, cudaStream_t s) {
    constexpr int E = N >= 256 ? 8 : (N == 128 ? 4 : 2), T = N / E;
    const size_t smem = (size_t)N * sizeof(tw_t<R>) + (size_t)line_len<cx<R>, N>() * sizeof(cx<R>) + 64 * sizeof(double);
    auto kern = ark45_1d_kernel<R, N, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)p.npaths, T, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

int ark45_1d_elems(int n) { return n >= 256 ? 8 : (n == 128 ? 4 : 2); }

template <typename R> cudaError_t launch_ark45_1d(int n, const AdaptiveParams<R> &p, cudaStream_t s) {
    switch (n) {
        case 64: return ark_launch<R, 64>(p, s);
        case 128: return ark_launch<R, 128>(p, s);
        case 256: return ark_launch<R, 256>(p, s);
        case 512: return ark_launch<R, 512>(p, s);
        case 1024: return ark_launch<R, 1024>(p, s);
        case 2048: return ark_launch<R, 2048>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_ark45_1d<float>(int, const AdaptiveParams<float> &, cudaStream_t);
template cudaError_t launch_ark45_1d<double>(int, const AdaptiveParams<double> &, cudaStream_t);

}  // namespace xsde
