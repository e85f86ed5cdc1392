// rk4ip_0d.cu -- RK4IP for zero-dimensional problems (ordinary SDEs), one thread per path.
//
// XMDS2 (arXiv:1204.4255) Sec. 2.5: fixed-step RK4 for Wiener-driven SDEs in
// Stratonovich form, many independent paths; Sec. 2.6: with no transverse
// dimension the interaction-picture factor exp(L dt/2) is the scalar exp(c0 dt/2).
// The state lives in registers for the whole run; a Philox draw per step.
#include "kernels.h"

namespace xsde {
namespace {

constexpr int kThreads0D = 256;

template <typename R> __global__ void __launch_bounds__(kThreads0D) rk4ip_0d_kernel(const Params0D<R> p) {
    using V = cx<R>;
    __shared__ double red[2][kThreads0D / 32];
    const int64_t lp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = lp < p.npaths;
    const uint32_t gp = (uint32_t)(p.lt.path_offset + lp);
    V z = (active && XSDE_IN(lp, p.npaths, p.status)) ? p.psi[lp] : mk<V>(R(0), R(0));
    const V E = p.Ehalf;
    const R gdt = p.lt.gdt;
    const R sixth = R(1) / R(6), third = R(1) / R(3), half = R(0.5);
    const int idx0[3] = {0, 0, 0};
    const bool vtime = p.lt.pot == PM_TABLE && p.lt.V_nt > 1;
    const R Vstatic = vtime ? R(0) : potential(p.lt, 0, idx0, 0, 0);

    for (int64_t n = 0;; ++n) {
        if (p.sm.every > 0 && n % p.sm.every == 0) {
            const int64_t s = n / p.sm.every;
            const double m2 = active ? (double)cabs2(z) : 0.0;
            if (active) {
                const double v = (double)potential(p.lt, 0, idx0, 0, p.step0 + n);
                if ((p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path &&
                    XSDE_IN(s * p.npaths + lp, p.sm.nsamp * p.npaths, p.status)) {
                    double *pq = p.sm.per_path + 2 * (s * p.npaths + lp);
                    pq[0] = m2;
                    pq[1] = (p.sm.h0 + v) * m2 + 0.5 * p.sm.g * m2 * m2;
                }
                if (!isfinite(m2)) atomicOr(p.status, ST_NONFINITE);
            }
            if ((p.sm.which & (MOM_MOD2 | MOM_MOD4)) && p.sm.per_point && XSDE_IN(s, p.sm.nsamp, p.status)) {
                double a = warp_sum(m2), b = warp_sum(m2 * m2);
                if ((threadIdx.x & 31) == 0) {
                    red[0][threadIdx.x >> 5] = a;
                    red[1][threadIdx.x >> 5] = b;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    double sa = 0.0, sb = 0.0;
                    for (int w = 0; w < kThreads0D / 32; ++w) {
                        sa += red[0][w];
                        sb += red[1][w];
                    }
                    atomicAdd(p.sm.per_point + 2 * s, sa * p.sm.inv_paths);
                    atomicAdd(p.sm.per_point + 2 * s + 1, sb * p.sm.inv_paths);
                }
                __syncthreads();
            }
        }
        if (n == p.nsteps) break;
        const uint64_t sg = p.step0 + n;
        const R v = vtime ? (XSDE_IN(sg, p.lt.V_nt, p.status) ? p.lt.V[sg] : R(0)) : Vstatic;
        const PointTerm<R> pt = point_term(p.lt, v, 0u, gp, (uint32_t)sg);
        if (p.scheme == 1) {
            // semi-implicit midpoint: a_I = D a; m <- a_I + N(m)/2 (three times); a <- D(2m - a_I)
            const V aI = cmul(E, z);
            V m = aI;
            for (int it = 0; it < 3; ++it) m = caxpy(aI, half, apply_N(m, pt, gdt));
            z = cmul(E, mk<V>(R(2) * m.x - aI.x, R(2) * m.y - aI.y));
            continue;
        }
        // a_I = D a, k1 = D N(a), k2, k3, k4 = N(D(a_I + k3)), a <- D(acc) + k4/6
        const V aI = cmul(E, z);
        const V k1 = cmul(E, apply_N(z, pt, gdt));
        const V k2 = apply_N(caxpy(aI, half, k1), pt, gdt);
        const V k3 = apply_N(caxpy(aI, half, k2), pt, gdt);
        const V k4 = apply_N(cmul(E, cadd(aI, k3)), pt, gdt);
        const V acc = caxpy(caxpy(caxpy(aI, sixth, k1), third, k2), third, k3);
        z = caxpy(cmul(E, acc), sixth, k4);
    }
    if (active && XSDE_IN(lp, p.npaths, p.status)) p.psi[lp] = z;
}

}  // namespace

template <typename R> cudaError_t launch_rk4ip_0d(const Params0D<R> &p, cudaStream_t s) {
    const int64_t blocks = (p.npaths + kThreads0D - 1) / kThreads0D;
    rk4ip_0d_kernel<R><<<(unsigned)blocks, kThreads0D, 0, s>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_rk4ip_0d<float>(const Params0D<float> &, cudaStream_t);
template cudaError_t launch_rk4ip_0d<double>(const Params0D<double> &, cudaStream_t);

}  // namespace xsde
