// rk4ip_adjoint.cu -- gradient of a final-state fidelity with respect to a
// space-time potential, through the discrete RK4IP scheme (1D lattices).
//
// Loss L = sum_p 1 - |<target|psi_N>|^2, <a|b> = sum conj(a) b dx, for the
// deterministic equation d psi/dt = L psi - i (V(x, t_n) + g|psi|^2) psi
// (XMDS2 Sec. 2.6, Eq. NonlinearSchrodingerEquationDimensionless with a
// time-dependent trap; the step of Sec. 2.5/2.6 as in rk4ip_1d.cu).
// Reverse mode on real vectors (Re, Im) with <u, v> = Re sum conj(u) v:
//   N(u) = dt(-i(V + g|u|^2)u) has tangent A du + B conj(du), A = -i dt (V + 2g|u|^2),
//   B = -i dt g u^2, adjoint mu -> conj(A) mu + B conj(mu); D^T = F^-1 conj(E) F;
//   dN/dV_j = -i dt u_j, so a stage with cotangent mu adds dt (mu.x u.y - mu.y u.x)
//   to dL/dV_j.
// A forward sweep keeps a checkpoint every K steps; every segment but the last
// is then recomputed from its checkpoint with the four stage inputs of each
// step (a, a_I + k1/2, a_I + k2/2, D(a_I + k3)) stored, and the reverse steps
// consume them.  Every transform pair runs on two vectors in lockstep, so a
// reverse step costs about one forward step.  Two schedules (AdjParams::phase):
//  - ADJ_FORWARD, ADJ_RECOMPUTE, ADJ_REVERSE: three launches.  The forward
//    sweep (one CTA per path) also stores the last segment's stage inputs and
//    the final state; all other segments are recomputed at once, one CTA per
//    (segment, path); the reverse sweep (one CTA per path) starts from the final
//    state.  Stage inputs of all steps are kept ([paths][nsteps][4][N]).
//  - ADJ_SEQUENTIAL: one launch, one CTA per path, recomputing one segment at a
//    time into a [paths][K][4][N] buffer (when the full buffer does not fit).
#include "fft.cuh"
#include "kernels.h"

namespace xsde {
namespace {

template <typename R> struct AdjMath {
    using V = cx<R>;
    // conj(A) mu + B conj(mu) at input u; dtV = dt (V + alpha xi), gdt = dt g
    __device__ __forceinline__ static V adjN(V u, V mu, R dtV, R gdt) {
        const R s = dtV + R(2) * gdt * cabs2(u);            // conj(A) = i s
        const R bx = gdt * R(2) * u.x * u.y;                  // B = gdt (2 ux uy, -(ux^2 - uy^2))
        const R by = -gdt * (u.x * u.x - u.y * u.y);
        return mk<V>(-s * mu.y + bx * mu.x + by * mu.y, s * mu.x + by * mu.x - bx * mu.y);
    }
    // Re(conj(mu) (-i dt u)) / dt
    __device__ __forceinline__ static R dv(V mu, V u) { return mu.x * u.y - mu.y * u.x; }
};

template <typename R, int N, int E>
__global__ void __launch_bounds__(N / E) rk4ip_adjoint_kernel(const AdjParams<R> p) {
    using V = cx<R>;
    using M = AdjMath<R>;
    constexpr int T = N / E;
    constexpr int BUF = line_len<V, N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tw_t<R> *tws = reinterpret_cast<tw_t<R> *>(smem_raw);
    V *bufA = reinterpret_cast<V *>(tws + N);
    V *bufB = bufA + BUF;
    double *red = reinterpret_cast<double *>(bufB + BUF);
    V *const sm2[2] = {bufA, bufB};
    const SyncBlock sync{};
    const TwiddleTable<tw_t<R>> tw{tws};
    const LineLayout<V> L{};
    const int t = threadIdx.x;
    const int64_t path = blockIdx.x;
    if (!XSDE_IN(path, p.npaths, p.status)) return;   // whole CTA: one path each
    const int64_t nck = (p.nsteps + p.K - 1) / p.K;    // checkpoints held by p.ckpt

    for (int i = t; i < N; i += blockDim.x) tws[i] = p.tw[i];
    __syncthreads();

    V Ek[E], El[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        Ek[m] = p.Etab[t + m * T];
        El[m] = p.Etab[N + t + m * T];
    }
    const R gdt = p.lt.gdt, dt = p.lt.dt;
    const R sixth = R(1) / R(6), third = R(1) / R(3), half = R(0.5);
    const bool vtime = p.lt.pot == PM_TABLE && p.lt.V_nt > 1;
    auto dtV_at = [&](int m, int64_t n) -> R {
        const int j = t + m * T;
        const int idx[3] = {j, 0, 0};
        return dt * (vtime ? p.lt.V[n * N + j] : potential(p.lt, 1, idx, j, 0));
    };
    auto nl = [&](V u, R dtv) -> V {   // N(u) = dt(-i(V + g|u|^2)u)
        const R s = dtv + gdt * cabs2(u);
        return mk<V>(s * u.y, -s * u.x);
    };
    // D (S = -1 then +1 with E) or its adjoint (conj(E)) on both vectors
    auto Dpair = [&](V (&x)[2][E], bool adjoint) {
        fft<N, E, -1, 2>(x, t, sm2, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            if (adjoint) {
                x[0][m] = cmulconj_hilo(x[0][m], Ek[m], El[m]);
                x[1][m] = cmulconj_hilo(x[1][m], Ek[m], El[m]);
            } else {
                x[0][m] = cmul_hilo(x[0][m], Ek[m], El[m]);
                x[1][m] = cmul_hilo(x[1][m], Ek[m], El[m]);
            }
        }
        fft<N, E, +1, 2>(x, t, sm2, L, sync, tw);
    };
    const size_t stride = (size_t)p.npaths * N;              // one field of all paths
    const bool full = p.phase != ADJ_SEQUENTIAL;
    // stage inputs of this path: [nsteps][4][N] (full) or [K][4][N]
    V *interm = p.interm + (size_t)path * (full ? p.nsteps : p.K) * 4 * N;
    // one forward step from x[0]; with `store`, keeps the stage inputs of step n
    auto forward = [&](V (&x)[2][E], int64_t n, bool store_in, int64_t slot) {
        const bool store = store_in && XSDE_IN(slot, p.interm_steps, p.status);
        R dtv[E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            dtv[m] = dtV_at(m, n);
            if (store) interm[(slot * 4 + 0) * N + t + m * T] = x[0][m];
            x[1][m] = nl(x[0][m], dtv[m]);
        }
        Dpair(x, false);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const V aI = x[0][m], k1 = x[1][m];
            const V w2 = caxpy(aI, half, k1);
            const V k2 = nl(w2, dtv[m]);
            const V w3 = caxpy(aI, half, k2);
            const V k3 = nl(w3, dtv[m]);
            if (store) {
                interm[(slot * 4 + 1) * N + t + m * T] = w2;
                interm[(slot * 4 + 2) * N + t + m * T] = w3;
            }
            x[0][m] = cadd(aI, k3);
            x[1][m] = caxpy(caxpy(caxpy(aI, sixth, k1), third, k2), third, k3);
        }
        Dpair(x, false);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            if (store) interm[(slot * 4 + 3) * N + t + m * T] = x[0][m];
            x[0][m] = caxpy(x[1][m], sixth, nl(x[0][m], dtv[m]));
        }
    };

    const int64_t nseg = (p.nsteps + p.K - 1) / p.K;
    const int64_t last0 = (nseg - 1) * p.K;
    V x[2][E];

    // ---- recomputation of segment blockIdx.y from its checkpoint ------------
    if (p.phase == ADJ_RECOMPUTE) {
        const int64_t n0 = (int64_t)blockIdx.y * p.K, n1 = n0 + p.K;   // never the last segment
        if (!XSDE_IN(blockIdx.y, nck, p.status)) return;
#pragma unroll
        for (int m = 0; m < E; ++m) x[0][m] = p.ckpt[blockIdx.y * stride + path * N + t + m * T];
        for (int64_t n = n0; n < n1; ++n) forward(x, n, true, n);
        return;
    }

    // ---- forward sweep with checkpoints ------------------------------------
    if (p.phase == ADJ_REVERSE) {
#pragma unroll
        for (int m = 0; m < E; ++m) x[0][m] = p.final_state[path * N + t + m * T];
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) x[0][m] = p.psi0[path * N + t + m * T];
        // the last segment keeps its stage inputs right away: the reverse
        // sweep starts there and needs no recomputation of it
        for (int64_t n = 0; n < p.nsteps; ++n) {
            if (n % p.K == 0 && XSDE_IN(n / p.K, nck, p.status)) {
#pragma unroll
                for (int m = 0; m < E; ++m) p.ckpt[(n / p.K) * stride + path * N + t + m * T] = x[0][m];
            }
            forward(x, n, n >= last0, full ? n : n - last0);
        }
        if (p.phase == ADJ_FORWARD) {
#pragma unroll
            for (int m = 0; m < E; ++m) p.final_state[path * N + t + m * T] = x[0][m];
            return;
        }
    }

    // ---- loss and the final cotangent ----------------------------------------
    double cr = 0.0, ci = 0.0;
    V tg[E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        tg[m] = p.target[t + m * T];
        const V a = x[0][m];     // conj(tg) a
        cr += (double)tg[m].x * a.x + (double)tg[m].y * a.y;
        ci += (double)tg[m].x * a.y - (double)tg[m].y * a.x;
    }
    cr = warp_sum(cr);
    ci = warp_sum(ci);
    if ((t & 31) == 0) {
        red[2 * (t >> 5)] = cr;
        red[2 * (t >> 5) + 1] = ci;
    }
    __syncthreads();
    cr = 0.0;
    ci = 0.0;
    for (int w = 0; w < T / 32; ++w) {   // T = N/8 >= 32 for the supported lengths
        cr += red[2 * w];
        ci += red[2 * w + 1];
    }
    cr *= p.dx;
    ci *= p.dx;
    if (t == 0) atomicAdd(p.loss, 1.0 - (cr * cr + ci * ci));
    // lambda_N = -2 c target dx
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const double lr = -2.0 * p.dx * (cr * tg[m].x - ci * tg[m].y);
        const double li = -2.0 * p.dx * (cr * tg[m].y + ci * tg[m].x);
        x[0][m] = mk<V>((R)lr, (R)li);
    }

    // ---- reverse sweep, segment by segment -----------------------------------
    V lam[E];
#pragma unroll
    for (int m = 0; m < E; ++m) lam[m] = x[0][m];
    for (int64_t sgi = nseg - 1; sgi >= 0; --sgi) {
        const int64_t n0 = sgi * p.K;
        const int64_t n1 = (n0 + p.K < p.nsteps) ? n0 + p.K : p.nsteps;
        if (!full && sgi != nseg - 1 && XSDE_IN(sgi, nck, p.status)) {
#pragma unroll
            for (int m = 0; m < E; ++m) x[0][m] = p.ckpt[sgi * stride + path * N + t + m * T];
            for (int64_t n = n0; n < n1; ++n) forward(x, n, true, n - n0);
        }
        for (int64_t n = n1 - 1; n >= n0; --n) {
            const int64_t slot = full ? n : n - n0;
            if (!XSDE_IN(slot, p.interm_steps, p.status) || !XSDE_IN(n, p.nsteps, p.status)) break;
            R dtv[E], gv[E];
            V y[2][E], w2s[E], w3s[E];
#pragma unroll
            for (int m = 0; m < E; ++m) {
                // FP64: the later stage inputs are fetched now so their latency
                // hides behind the first transform pair (FP32 fetches them late:
                // the extra live registers cost more than the latency there)
                if constexpr (sizeof(R) == 8) {
                    w2s[m] = interm[(slot * 4 + 1) * N + t + m * T];
                    w3s[m] = interm[(slot * 4 + 2) * N + t + m * T];
                }
                dtv[m] = dtV_at(m, n);
                const V Du1 = interm[(slot * 4 + 3) * N + t + m * T];
                const V l4 = cscale(lam[m], sixth);
                y[0][m] = lam[m];
                y[1][m] = M::adjN(Du1, l4, dtv[m], gdt);
                gv[m] = M::dv(l4, Du1);
            }
            Dpair(y, true);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const V w2 = (sizeof(R) == 8) ? w2s[m] : interm[(slot * 4 + 1) * N + t + m * T];
                const V w3 = (sizeof(R) == 8) ? w3s[m] : interm[(slot * 4 + 2) * N + t + m * T];
                const V la = y[0][m], lu = y[1][m];
                const V lk3 = caxpy(lu, third, la);
                const V lw3 = M::adjN(w3, lk3, dtv[m], gdt);
                gv[m] += M::dv(lk3, w3);
                const V lk2 = caxpy(cscale(la, third), half, lw3);
                const V lw2 = M::adjN(w2, lk2, dtv[m], gdt);
                gv[m] += M::dv(lk2, w2);
                y[0][m] = caxpy(cscale(la, sixth), half, lw2);        // lambda_k1
                y[1][m] = cadd(cadd(cadd(la, lu), lw3), lw2);          // lambda_aI
            }
            Dpair(y, true);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const V a = interm[(slot * 4 + 0) * N + t + m * T];
                lam[m] = cadd(M::adjN(a, y[0][m], dtv[m], gdt), y[1][m]);
                gv[m] += M::dv(y[0][m], a);
                atomicAdd(p.dLdV + n * N + t + m * T, (double)(gv[m] * dt));
            }
        }
    }
    if (p.dLdpsi0) {
#pragma unroll
        for (int m = 0; m < E; ++m) p.dLdpsi0[path * N + t + m * T] = lam[m];
    }
}

template <typename R, int N, int E> cudaError_t adj_launch(const AdjParams<R> &p, cudaStream_t s) {
    constexpr int T = N / E;
    const size_t smem = (size_t)N * sizeof(tw_t<R>) + (size_t)2 * line_len<cx<R>, N>() * sizeof(cx<R>) +
                        (size_t)2 * ((T + 31) / 32) * sizeof(double);
    auto kern = rk4ip_adjoint_kernel<R, N, E>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned segs = (unsigned)((p.nsteps + p.K - 1) / p.K);
    const dim3 grid((unsigned)p.npaths, p.phase == ADJ_RECOMPUTE ? segs - 1 : 1u);
    if (grid.y == 0) return cudaSuccess;     // a single segment: nothing to recompute
    kern<<<grid, T, smem, s>>>(p);
    return cudaGetLastError();
}

template <typename R, int N> cudaError_t adj_launch_e(int elems, const AdjParams<R> &p, cudaStream_t s) {
    return elems == 4 ? adj_launch<R, N, 4>(p, s) : adj_launch<R, N, 8>(p, s);
}

}  // namespace

// elems: points per thread, 8 (radix-8 plan) or 4 (radix-4 plan; p.tw must
// hold that plan's table)
template <typename R> cudaError_t launch_adjoint_1d(int n, int elems, const AdjParams<R> &p, cudaStream_t s) {
    switch (n) {
        case 256: return adj_launch_e<R, 256>(elems, p, s);
        case 512: return adj_launch_e<R, 512>(elems, p, s);
        case 1024: return adj_launch_e<R, 1024>(elems, p, s);
        case 2048: return adj_launch_e<R, 2048>(elems, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// XSDE_REAL_BITS selects one precision per translation unit (parallel builds)
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 32
template cudaError_t launch_adjoint_1d<float>(int, int, const AdjParams<float> &, cudaStream_t);
#endif
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 64
template cudaError_t launch_adjoint_1d<double>(int, int, const AdjParams<double> &, cudaStream_t);
#endif

}  // namespace xsde
