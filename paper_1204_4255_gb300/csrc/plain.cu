// plain.cu -- the unfused RK4IP step, for comparison with the fused passes.
//
// The same scheme as the fused kernels (XMDS2 Secs. 2.5-2.6: RK4 in the
// interaction picture re-centred each step), written the way a direct port of
// a CPU code would run it on a GPU: every transform is a cuFFT call over the
// whole batch, and every other operation -- exp(L dt/2) in Fourier space, the
// real-space term N(u) = dt g(u), each Runge-Kutta combination -- is its own
// elementwise kernel, so each intermediate field goes through HBM.  Per step:
//   a_I = D a,  k1 = D N(a),  k2 = N(a_I + k1/2),  k3 = N(a_I + k2/2),
//   k4 = N(D(a_I + k3)),  a <- D(a_I + k1/6 + k2/3 + k3/3) + k4/6,
// with D u = F^-1 [E F u] and E = exp(L(k) dt/2)/N_total tabulated at every k.
#include <new>

#include <cufft.h>

#include "kernels.h"

namespace xsde {
namespace {

constexpr int kThreads = 256;

unsigned grid_for(int64_t n, int num_sms) {
    const int64_t want = (n + kThreads - 1) / kThreads;
    const int64_t cap = (int64_t)num_sms * 16;
    return (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
}

// out = N(in) = dt g(in) at global step sg (the real-space term of the step)
template <typename R>
__global__ void __launch_bounds__(kThreads) plain_nonlinear(cx<R> *out, const cx<R> *in, const PlainParams<R> p,
                                                            uint64_t sg) {
    const int64_t total = p.npaths * p.npts;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t path = i / p.npts, j = i - path * p.npts;
        int idx[3] = {0, 0, 0};
        int64_t r = j;
        for (int d = p.ndim - 1; d >= 0; --d) {
            idx[d] = (int)(r % p.n[d]);
            r /= p.n[d];
        }
        const R v = potential(p.lt, p.ndim, idx, j, sg);
        const PointTerm<R> pt = point_term(p.lt, v, (uint32_t)j, (uint32_t)(p.lt.path_offset + path), (uint32_t)sg);
        out[i] = apply_N(in[i], pt, p.lt.gdt);
    }
}

// x <- E x in Fourier space
template <typename R>
__global__ void __launch_bounds__(kThreads) plain_mul_E(cx<R> *x, const cx<R> *E, int64_t npts, int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<R> e = E[i % npts], u = x[i];
        x[i] = mk<cx<R>>(u.x * e.x - u.y * e.y, u.x * e.y + u.y * e.x);
    }
}

// out = x + c k
template <typename R>
__global__ void __launch_bounds__(kThreads) plain_axpy(cx<R> *out, const cx<R> *x, const cx<R> *k, R c,
                                                       int64_t total) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const cx<R> a = x[i], b = k[i];
        out[i] = mk<cx<R>>(a.x + c * b.x, a.y + c * b.y);
    }
}

cudaError_t from_cufft(cufftResult r) {
    if (r == CUFFT_SUCCESS) return cudaSuccess;
    return r == CUFFT_ALLOC_FAILED ? cudaErrorMemoryAllocation : cudaErrorUnknown;
}

template <typename R> cudaError_t exec(cufftHandle h, cx<R> *x, int dir);
template <> cudaError_t exec<float>(cufftHandle h, cx<float> *x, int dir) {
    return from_cufft(cufftExecC2C(h, reinterpret_cast<cufftComplex *>(x), reinterpret_cast<cufftComplex *>(x), dir));
}
template <> cudaError_t exec<double>(cufftHandle h, cx<double> *x, int dir) {
    return from_cufft(
        cufftExecZ2Z(h, reinterpret_cast<cufftDoubleComplex *>(x), reinterpret_cast<cufftDoubleComplex *>(x), dir));
}

}  // namespace

struct PlainPlan {
    cufftHandle h = 0;
    bool fp64 = false;
    int ndim = 0;
    int n[3] = {0, 0, 0};
    int64_t npaths = 0;
};

cudaError_t plain_plan_create(int ndim, const int *n, int64_t npaths, bool fp64, PlainPlan **out) {
    *out = nullptr;
    PlainPlan *pl = new (std::nothrow) PlainPlan();
    if (!pl) return cudaErrorMemoryAllocation;
    int64_t npts = 1;
    for (int d = 0; d < ndim; ++d) {
        pl->n[d] = n[d];
        npts *= n[d];
    }
    pl->fp64 = fp64;
    pl->ndim = ndim;
    pl->npaths = npaths;
    int dims[3] = {n[0], ndim > 1 ? n[1] : 1, ndim > 2 ? n[2] : 1};
    const cufftResult r = cufftPlanMany(&pl->h, ndim, dims, nullptr, 1, (int)npts, nullptr, 1, (int)npts,
                                        fp64 ? CUFFT_Z2Z : CUFFT_C2C, (int)npaths);
    if (r != CUFFT_SUCCESS) {
        delete pl;
        return from_cufft(r);
    }
    *out = pl;
    return cudaSuccess;
}

void plain_plan_destroy(PlainPlan *pl) {
    if (!pl) return;
    cufftDestroy(pl->h);
    delete pl;
}

bool plain_plan_matches(const PlainPlan *pl, int ndim, const int *n, int64_t npaths, bool fp64) {
    if (!pl || pl->ndim != ndim || pl->npaths != npaths || pl->fp64 != fp64) return false;
    for (int d = 0; d < ndim; ++d)
        if (pl->n[d] != n[d]) return false;
    return true;
}

template <typename R> cudaError_t run_plain(PlainPlan *pl, const PlainParams<R> &p, int num_sms, cudaStream_t s) {
    using V = cx<R>;
    cudaError_t e = from_cufft(cufftSetStream(pl->h, s));
    if (e != cudaSuccess) return e;
    const int64_t total = p.npaths * p.npts;
    const unsigned grid = grid_for(total, num_sms);
    const size_t bytes = (size_t)total * sizeof(V);
    auto D = [&](V *x) -> cudaError_t {
        cudaError_t r = exec<R>(pl->h, x, CUFFT_FORWARD);
        if (r != cudaSuccess) return r;
        plain_mul_E<R><<<grid, kThreads, 0, s>>>(x, p.E, p.npts, total);
        if ((r = cudaGetLastError()) != cudaSuccess) return r;
        return exec<R>(pl->h, x, CUFFT_INVERSE);
    };
    auto N = [&](V *out, const V *in, uint64_t sg) -> cudaError_t {
        plain_nonlinear<R><<<grid, kThreads, 0, s>>>(out, in, p, sg);
        return cudaGetLastError();
    };
    auto axpy = [&](V *out, const V *x, const V *k, R c) -> cudaError_t {
        plain_axpy<R><<<grid, kThreads, 0, s>>>(out, x, k, c, total);
        return cudaGetLastError();
    };
#define XSDE_TRY(call)                          \
    do {                                        \
        if ((e = (call)) != cudaSuccess) return e; \
    } while (0)
    const R sixth = R(1) / R(6), third = R(1) / R(3), half = R(0.5);
    for (int64_t n = 0; n < p.nsteps; ++n) {
        const uint64_t sg = p.step0 + n;
        XSDE_TRY(cudaMemcpyAsync(p.aI, p.a, bytes, cudaMemcpyDeviceToDevice, s));
        XSDE_TRY(D(p.aI));                            // a_I = D a
        XSDE_TRY(N(p.k, p.a, sg));
        XSDE_TRY(D(p.k));                             // k1 = D N(a)
        XSDE_TRY(axpy(p.acc, p.aI, p.k, sixth));
        XSDE_TRY(axpy(p.tmp, p.aI, p.k, half));
        XSDE_TRY(N(p.k, p.tmp, sg));                  // k2
        XSDE_TRY(axpy(p.acc, p.acc, p.k, third));
        XSDE_TRY(axpy(p.tmp, p.aI, p.k, half));
        XSDE_TRY(N(p.k, p.tmp, sg));                  // k3
        XSDE_TRY(axpy(p.acc, p.acc, p.k, third));
        XSDE_TRY(axpy(p.tmp, p.aI, p.k, R(1)));
        XSDE_TRY(D(p.tmp));                           // D(a_I + k3)
        XSDE_TRY(D(p.acc));                           // D(a_I + k1/6 + k2/3 + k3/3)
        XSDE_TRY(N(p.k, p.tmp, sg));                  // k4
        XSDE_TRY(axpy(p.a, p.acc, p.k, sixth));
    }
#undef XSDE_TRY
    return cudaSuccess;
}

// XSDE_REAL_BITS selects one precision per translation unit (parallel builds)
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 32
template cudaError_t run_plain<float>(PlainPlan *, const PlainParams<float> &, int, cudaStream_t);
#endif
#if !defined(XSDE_REAL_BITS) || XSDE_REAL_BITS == 64
template cudaError_t run_plain<double>(PlainPlan *, const PlainParams<double> &, int, cudaStream_t);
#endif

}  // namespace xsde
