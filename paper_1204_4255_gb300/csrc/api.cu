// api.cu -- the C-ABI of include/xsde.h: handles, host-side validation, the
// Fourier-space tables, and the pass schedule of one xsde_integrate call.
//
// Tables (XMDS2 Sec. 2.6: only exp(+-L dt) factors are needed for fixed steps)
// are evaluated in FP64 on the host and rounded once to the working precision.
// FP32 rounding is chosen for what a long run accumulates:
//  - FFT twiddles: FP32 twiddles sit on average ~1e-8 below unit modulus at
//    the angles the early stages use, which drains the norm every transform;
//  - exp(L dt/2): applied to the same mode every step, so both phase and
//    modulus errors grow linearly with the step count.
// Both are therefore stored as FP32 hi + lo (lo = rounded remainder of the
// FP64 value) and applied with compensated FMAs (device_common.cuh).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/xsde.h"
#include "kernels.h"

using namespace xsde;

struct xsde_grid {
    int ndim;
    int n[3];
    double xmin[3], xmax[3];
    int64_t npts;
    int basis[3];   // XSDE_BASIS_* per dimension (xsde_grid_set_basis)
};

struct xsde_vector {
    xsde_grid grid;
    xsde_dtype dtype;
    int ncomp;
    int64_t npaths;
    void *data;
    bool owned;
};

struct xsde_noise {
    xsde_noise_kind kind;
    uint64_t seed;
};

struct xsde_problem {
    xsde_grid grid;
    xsde_dtype dtype;
    int device;
    bool have_ops = false;
    xsde_linear_op L{};
    xsde_nonlinear_op N{};
    xsde_noise noise{XSDE_NOISE_NONE, 0};
    xsde_sampling samp{0, 0};
    double *per_path = nullptr, *per_point = nullptr;
    double table_dt = -1.0;
    void *d_tw[3] = {nullptr, nullptr, nullptr};
    void *d_tw1d[2] = {nullptr, nullptr};   // 1D: twiddles of the radix-4 and radix-2 plans
    void *d_tw2[3] = {nullptr, nullptr, nullptr};   // complex64 2D/3D: two-stage plan twiddles (warp column pass)
    void *d_twp = nullptr;   // complex64 2D/3D: paired twiddles of the row dimension (TMA row pass)
    void *d_E[3] = {nullptr, nullptr, nullptr};
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    int *d_status = nullptr;
    int num_sms = 1;
    int kernel_variant = 0;   // see xsde_set_kernel_variant
    int noise_substeps = 1;   // see xsde_set_noise_substeps
    int scheme = XSDE_SCHEME_RK4IP;   // see xsde_set_scheme
    void *d_knl = nullptr;    // non-local kernel khat/npts in the problem's precision [npts]
    void *d_B = nullptr;      // cosine / sine dimension 0: the B table of its pair step
    void *d_B1 = nullptr;     // cosine / sine dimension 1: the B table of its pair step
    void *d_B2 = nullptr;     // cosine / sine dimension 2 of a 3D lattice: the B table of its pair step
    void *d_Ef[3] = {nullptr, nullptr, nullptr};   // whole-step factors exp(L dt) per dimension (2D/3D semi-implicit)
    bool nonlocal = false;    // see xsde_set_nonlocal
    uint64_t generation = 0;  // bumped by every call that changes what integrate launches
    void *d_adj = nullptr;    // adjoint checkpoints and stage inputs
    size_t adj_bytes = 0;
    // unfused comparison path (xsde_integrate_plain)
    PlainPlan *plain = nullptr;
    void *d_plain = nullptr;  // four work fields
    size_t plain_bytes = 0;
    void *d_plain_E = nullptr;  // exp(L dt/2)/npts at every k
    void *d_hostfield = nullptr;  // device copy of a host field (xsde_integrate_host)
    size_t hostfield_bytes = 0;
    double plain_dt = -1.0;
    uint64_t plain_gen = ~0ull;
    // launch profiling: CUDA events around every kernel launch of this problem
    bool profiling = false;
    struct Mark {
        int kind;
        cudaEvent_t start, stop;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[XSDE_KERNEL_KINDS] = {};
    int64_t prof_launches[XSDE_KERNEL_KINDS] = {};
};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? XSDE_ENOMEM : XSDE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define XSDE_CUDA(call, what)                        \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool pow2_in_range(int n) { return n >= 16 && n <= 2048 && (n & (n - 1)) == 0; }

const char *const kKernelNames[XSDE_KERNEL_KINDS] = {
    "rk4ip_0d",      "rk4ip_1d",      "row_prologue", "row_stage2", "row_steady",
    "row_epilogue",  "row_fft_only",  "col_propagate", "col_spectral", "row_nonlocal",
    "col_convolve"};

cudaEvent_t take_event(xsde_problem *p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch through `fn` and, when profiling, bracket it with events on stream s.
// NVTX ranges named after the kernel kinds around every launch, for timeline
// tools, when the environment sets XSDE_NVTX=1 (read once)
bool nvtx_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("XSDE_NVTX");
        return v && v[0] == '1';
    }();
    return on;
}

template <typename F> cudaError_t launch_ranged(int kind, F &&fn) {
    if (!nvtx_enabled()) return fn();
    nvtxRangePushA(kind >= 0 && kind < XSDE_KERNEL_KINDS ? kKernelNames[kind] : "xsde");
    cudaError_t e = fn();
    nvtxRangePop();
    return e;
}

template <typename F> cudaError_t timed(xsde_problem *p, int kind, cudaStream_t s, F &&fn) {
    if (!p->profiling) return launch_ranged(kind, fn);
    cudaEvent_t a = take_event(p), b = take_event(p);
    if (a) cudaEventRecord(a, s);
    cudaError_t e = launch_ranged(kind, fn);
    if (b) cudaEventRecord(b, s);
    if (a && b) p->marks.push_back({kind, a, b});
    return e;
}

// Fold finished event pairs into the per-kind totals (after a synchronize).
void collect_marks(xsde_problem *p) {
    for (auto &m : p->marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.start, m.stop) == cudaSuccess) {
            p->prof_ms[m.kind] += ms;
            p->prof_launches[m.kind] += 1;
        }
        p->event_pool.push_back(m.start);
        p->event_pool.push_back(m.stop);
    }
    p->marks.clear();
}

size_t elem_bytes(xsde_dtype d) { return d == XSDE_C64 ? 8 : 16; }

double grid_dx(const xsde_grid &g, int d) { return (g.xmax[d] - g.xmin[d]) / g.n[d]; }
double grid_dV(const xsde_grid &g) {
    double v = 1.0;
    for (int d = 0; d < g.ndim; ++d) v *= grid_dx(g, d);
    return v;
}
bool any_basis(const xsde_grid &g) {
    for (int d = 0; d < g.ndim; ++d)
        if (g.basis[d] != XSDE_BASIS_FOURIER) return true;
    return false;
}
// wavenumber of spectral index i along d: Fourier k = 2 pi m/L (m = i or i - n);
// cosine k = pi i/L; sine k = pi (i+1)/L
double kval(const xsde_grid &g, int d, int i) {
    const int n = g.n[d];
    const double len = g.xmax[d] - g.xmin[d];
    if (g.basis[d] == XSDE_BASIS_COS) return M_PI * i / len;
    if (g.basis[d] == XSDE_BASIS_SIN) return M_PI * (i + 1) / len;
    return 2.0 * M_PI / len * (i < n / 2 ? i : i - n);
}

// A cosine / sine dimension applies the diagonal factors f of its modes
// through the FFT of its even-odd ordered points: U_k = A_k V_k + B_k V_{n-k},
// A_k = (F_k + F_{n-k})/2, B_k = exp(i pi k/n) (F_k - F_{n-k})/2 (A_0 = F_0,
// B_0 = 0) with F the cosine factors in mode order, or for the sine basis the
// sine factors reversed (F_k = f_{n-1-k}).
void trig_pair_tables(int basis, const std::vector<std::complex<double>> &f, std::vector<std::complex<double>> &A,
                      std::vector<std::complex<double>> &B) {
    const int n = (int)f.size();
    std::vector<std::complex<double>> F(n);
    for (int k = 0; k < n; ++k) F[k] = basis == XSDE_BASIS_SIN ? f[n - 1 - k] : f[k];
    A.assign(n, 0.0);
    B.assign(n, 0.0);
    A[0] = F[0];
    for (int k = 1; k < n; ++k) {
        A[k] = 0.5 * (F[k] + F[n - k]);
        B[k] = 0.5 * std::polar(1.0, M_PI * k / n) * (F[k] - F[n - k]);
    }
}

// value -> hi (nearest) and lo (nearest to the remainder); FP64 keeps lo = 0
void split_hi_lo(const std::complex<double> &z, float2 *hi, float2 *lo) {
    const float hr = (float)z.real(), hm = (float)z.imag();
    *hi = make_float2(hr, hm);
    *lo = make_float2((float)(z.real() - (double)hr), (float)(z.imag() - (double)hm));
}
void split_hi_lo(const std::complex<double> &z, double2 *hi, double2 *lo) {
    *hi = make_double2(z.real(), z.imag());
    *lo = make_double2(0.0, 0.0);
}

template <typename V> int upload_raw(const std::vector<V> &tmp, void **dptr, cudaStream_t s) {
    if (!*dptr) XSDE_CUDA(cudaMalloc(dptr, tmp.size() * sizeof(V)), "cudaMalloc(table)");
    XSDE_CUDA(cudaMemcpyAsync(*dptr, tmp.data(), tmp.size() * sizeof(V), cudaMemcpyHostToDevice, s),
              "cudaMemcpyAsync(table)");
    XSDE_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize(table)");
    return XSDE_OK;
}

// twiddle table exp(-2 pi i m/n), m < n: FP64 (cos, sin); FP32 (hi, lo) split
void make_twiddle(const std::complex<double> &z, double2 *out) { *out = make_double2(z.real(), z.imag()); }
void make_twiddle(const std::complex<double> &z, float4 *out) {
    float2 hi, lo;
    split_hi_lo(z, &hi, &lo);
    *out = make_float4(hi.x, hi.y, lo.x, lo.y);
}

// the paired form (c, s, c eps, s eps) of a twiddle for fft.cuh's fftp_* and
// fft2.cuh: (c, s) its FP32 rounding, eps = 1/(c^2 + s^2) - 1, the part that
// makes the backward transform the exact inverse of the forward
void make_twiddle_paired(const std::complex<double> &z, float4 *out) {
    const float c = (float)z.real(), sn = (float)z.imag();
    const double eps = 1.0 / ((double)c * c + (double)sn * sn) - 1.0;
    *out = make_float4(c, sn, (float)(c * eps), (float)(sn * eps));
}

// per-stage layout of fft.cuh: stage (Ns, R) holds w_n^(r k n/(Ns R)) at
// [stage_table_offset(n, Ns) + (r-1) Ns + k]; n entries are allocated (the
// table needs at most n - 1).  PAIRED (complex64): entries for fftp_*.
template <typename R, int E = 8, bool PAIRED = false> int upload_twiddles(int n, void **dptr, cudaStream_t s) {
    std::vector<tw_t<R>> tmp(n);
    auto put = [&](const std::complex<double> &z, tw_t<R> *out) {
        if constexpr (PAIRED) make_twiddle_paired(z, out);
        else make_twiddle(z, out);
    };
    put(std::complex<double>(0.0, 0.0), &tmp[n - 1]);
    for (int ns = 1; ns < n;) {
        const int rad = stage_radix<E>(n / ns);
        if (ns > 1) {
            const int off = stage_table_offset<E>(n, ns);
            for (int r = 1; r < rad; ++r)
                for (int k = 0; k < ns; ++k) {
                    const long m = (long)r * k * (n / (ns * rad));
                    put(std::polar(1.0, -2.0 * M_PI * (double)m / n), &tmp[off + (r - 1) * ns + k]);
                }
        }
        ns *= rad;
    }
    return upload_raw(tmp, dptr, s);
}

// twiddles of the two-stage plan of fft2.cuh (E points per lane): entry
// (r-1) E + j holds w_n^(r j), r in [1, n/E), j in [0, E)
int upload_twiddles_2stage(int n, int E, void **dptr, cudaStream_t s) {
    std::vector<float4> tmp((size_t)(n / E - 1) * E);
    for (int r = 1; r < n / E; ++r)
        for (int j = 0; j < E; ++j)
            make_twiddle_paired(std::polar(1.0, -2.0 * M_PI * (double)((long)r * j) / n), &tmp[(size_t)(r - 1) * E + j]);
    return upload_raw(tmp, dptr, s);
}

// factor table as [hi[0..n), lo[0..n)]
template <typename V> int upload(const std::vector<std::complex<double>> &h, void **dptr, cudaStream_t s) {
    const size_t n = h.size();
    std::vector<V> tmp(2 * n);
    for (size_t i = 0; i < n; ++i) split_hi_lo(h[i], &tmp[i], &tmp[n + i]);
    return upload_raw(tmp, dptr, s);
}

// twiddles and the exp(L dt/2) factors for this dt
template <typename V> int ensure_tables(xsde_problem *p, double dt, cudaStream_t s) {
    if (p->table_dt == dt) return XSDE_OK;
    const xsde_grid &g = p->grid;
    const std::complex<double> c0(p->L.c0_re, p->L.c0_im), c2(p->L.c2_re, p->L.c2_im);
    int rc;
    for (int d = 0; d < g.ndim; ++d)
        if ((rc = upload_twiddles<decltype(V::x)>(g.n[d], &p->d_tw[d], s)) != XSDE_OK) return rc;
    if constexpr (std::is_same<V, float2>::value) {
        for (int d = 0; d < g.ndim && g.ndim >= 2; ++d)
            if (warp_col_supported(g.n[d], WARP_COL_C) &&
                (rc = upload_twiddles_2stage(g.n[d], warp_col_elems(g.n[d]), &p->d_tw2[d], s)) != XSDE_OK)
                return rc;
        if (g.ndim >= 2 && tma_row_supported(g.n[g.ndim - 1]) &&
            (rc = upload_twiddles<float, 8, true>(g.n[g.ndim - 1], &p->d_twp, s)) != XSDE_OK)
            return rc;
    }
    if (g.ndim == 1) {
        const int n = g.n[0];
        // the radix-4 and radix-2 plans of the 4- and 2-element launch shapes
        if ((rc = upload_twiddles<decltype(V::x), 4>(n, &p->d_tw1d[0], s)) != XSDE_OK) return rc;
        if ((rc = upload_twiddles<decltype(V::x), 2>(n, &p->d_tw1d[1], s)) != XSDE_OK) return rc;
        std::vector<std::complex<double>> e(n);
        for (int i = 0; i < n; ++i) {
            const double k = kval(g, 0, i);
            e[i] = std::exp((c0 + c2 * (k * k)) * (0.5 * dt)) / (double)n;
        }
        if (g.basis[0] != XSDE_BASIS_FOURIER) {
            std::vector<std::complex<double>> A, B;
            trig_pair_tables(g.basis[0], e, A, B);
            if ((rc = upload<V>(A, &p->d_E[0], s)) != XSDE_OK) return rc;
            if ((rc = upload<V>(B, &p->d_B, s)) != XSDE_OK) return rc;
        } else if ((rc = upload<V>(e, &p->d_E[0], s)) != XSDE_OK) {
            return rc;
        }
    } else if (g.ndim == 2) {
        const int n0 = g.n[0];
        std::vector<std::complex<double>> e0(n0), e1(g.n[1]);
        for (int i = 0; i < n0; ++i) {
            const double k = kval(g, 0, i);
            e0[i] = std::exp((c0 + c2 * (k * k)) * (0.5 * dt)) / ((double)n0 * g.n[1]);
        }
        if (g.basis[0] != XSDE_BASIS_FOURIER) {
            std::vector<std::complex<double>> A, B;
            trig_pair_tables(g.basis[0], e0, A, B);
            e0 = A;
            if ((rc = upload<V>(B, &p->d_B, s)) != XSDE_OK) return rc;
        }
        for (int i = 0; i < g.n[1]; ++i) {
            const double k = kval(g, 1, i);
            e1[i] = std::exp(c2 * (k * k) * (0.5 * dt));
        }
        if (g.basis[1] != XSDE_BASIS_FOURIER) {
            std::vector<std::complex<double>> A, B;
            trig_pair_tables(g.basis[1], e1, A, B);
            e1 = A;
            if ((rc = upload<V>(B, &p->d_B1, s)) != XSDE_OK) return rc;
        }
        if ((rc = upload<V>(e0, &p->d_E[0], s)) != XSDE_OK) return rc;
        if ((rc = upload<V>(e1, &p->d_E[1], s)) != XSDE_OK) return rc;
        if (p->scheme == XSDE_SCHEME_SEMI_IMPLICIT) {
            // a whole step exp(L dt) between two semi-implicit stages (no pairing: Fourier lattices)
            std::vector<std::complex<double>> f0(g.n[0]), f1(g.n[1]);
            for (int i = 0; i < g.n[0]; ++i) {
                const double k = kval(g, 0, i);
                f0[i] = std::exp((c0 + c2 * (k * k)) * dt) / ((double)g.n[0] * g.n[1]);
            }
            for (int i = 0; i < g.n[1]; ++i) {
                const double k = kval(g, 1, i);
                f1[i] = std::exp(c2 * (k * k) * dt);
            }
            if ((rc = upload<V>(f0, &p->d_Ef[0], s)) != XSDE_OK) return rc;
            if ((rc = upload<V>(f1, &p->d_Ef[1], s)) != XSDE_OK) return rc;
        }
    } else if (g.ndim == 3) {
        // exp(L dt/2) = E0(k0) E1(k1) E2(k2); E0 carries exp(c0 dt/2)/(n0 n1 n2)
        // (and, for the semi-implicit step, the same for the whole step exp(L dt))
        const int nh = p->scheme == XSDE_SCHEME_SEMI_IMPLICIT ? 2 : 1;
        for (int h = 0; h < nh; ++h) {
            const double tau = h == 0 ? 0.5 * dt : dt;
            for (int d = 0; d < 3; ++d) {
                std::vector<std::complex<double>> e(g.n[d]);
                for (int i = 0; i < g.n[d]; ++i) {
                    const double k = kval(g, d, i);
                    e[i] = d == 0 ? std::exp((c0 + c2 * (k * k)) * tau) / ((double)g.n[0] * g.n[1] * g.n[2])
                                  : std::exp(c2 * (k * k) * tau);
                }
                if (h == 0 && g.basis[d] != XSDE_BASIS_FOURIER) {
                    // a cosine / sine dimension: the A table in E[d], the B table beside it
                    std::vector<std::complex<double>> A, B;
                    trig_pair_tables(g.basis[d], e, A, B);
                    e = A;
                    if ((rc = upload<V>(B, d == 0 ? &p->d_B : d == 1 ? &p->d_B1 : &p->d_B2, s)) != XSDE_OK) return rc;
                }
                if ((rc = upload<V>(e, h == 0 ? &p->d_E[d] : &p->d_Ef[d], s)) != XSDE_OK) return rc;
            }
        }
    }
    p->table_dt = dt;
    return XSDE_OK;
}

template <typename R>
void fill_terms(const xsde_problem *p, double dt, int64_t npaths, int64_t path_offset, LocalTerm<R> &lt,
                Sampling &sm) {
    const xsde_grid &g = p->grid;
    const double dV = grid_dV(g);
    lt.dt = (R)dt;
    lt.gdt = (R)(p->N.g * dt);
    lt.pot = p->N.pot_kind;
    for (int d = 0; d < 3; ++d) {
        lt.hw2[d] = (R)(d < g.ndim ? 0.5 * p->N.omega[d] * p->N.omega[d] : 0.0);
        // cosine / sine lattices are cell-centred: x_j = xmin + (j + 1/2) dx
        lt.xmin[d] = (R)(d < g.ndim ? g.xmin[d] + (g.basis[d] ? 0.5 * grid_dx(g, d) : 0.0) : 0.0);
        lt.dx[d] = (R)(d < g.ndim ? grid_dx(g, d) : 0.0);
    }
    lt.V = static_cast<const R *>(p->N.V);
    lt.V_nt = p->N.V_nt;
    lt.npts = g.npts;
    lt.noise = NM_NONE;
    lt.nscale = 0;
    if (p->noise.kind != XSDE_NOISE_NONE) {
        const double base = p->N.amplitude * std::sqrt(dt / dV);
        if (p->N.coupling == XSDE_COUPLE_MULTIPLICATIVE) {
            lt.noise = NM_MUL_REAL;
            lt.nscale = (R)base;
        } else if (p->noise.kind == XSDE_NOISE_WIENER_REAL) {
            lt.noise = NM_ADD_REAL;
            lt.nscale = (R)base;
        } else {
            lt.noise = NM_ADD_COMPLEX;
            lt.nscale = (R)(base / std::sqrt(2.0));
        }
    }
    lt.key = make_uint2((uint32_t)(p->noise.seed & 0xffffffffu), (uint32_t)(p->noise.seed >> 32));
    lt.path_offset = path_offset;
    lt.substeps = p->noise_substeps;
    lt.status = p->d_status;

    sm.every = p->samp.every;
    sm.which = p->samp.which;
    sm.per_path = p->per_path;
    sm.per_point = p->per_point;
    sm.dV = dV;
    sm.inv_paths = 1.0 / (double)npaths;
    sm.h0 = -p->L.c0_im;
    sm.h2 = -p->L.c2_im;
    for (int d = 0; d < 3; ++d)
        sm.kscale[d] = d < g.ndim ? (g.basis[d] ? M_PI : 2.0 * M_PI) / (g.xmax[d] - g.xmin[d]) : 0.0;
    sm.g = p->N.g;
}

// cuTensorMapEncodeTiled from the driver, fetched once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }();
    return fn;
}

// A complex64 field viewed as [rows][cols] 8-byte elements for the column
// pass: box COL_TMA_C x col_tma_box_rows(n0) (n0 = the column length).
bool encode_field_map(CUtensorMap *m, void *base, int64_t rows, int64_t cols, int n0) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
    cuuint32_t box[2] = {(cuuint32_t)COL_TMA_C, (cuuint32_t)col_tma_box_rows(n0)};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same view for the warp column pass: box WARP_COL_C x warp_col_box_rows(n0)
// (64-byte rows), written to shared memory with the 64-byte swizzle.
bool encode_field_map_warp(CUtensorMap *m, void *base, int64_t rows, int64_t cols, int n0) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
    cuuint32_t box[2] = {(cuuint32_t)WARP_COL_C, (cuuint32_t)warp_col_box_rows(n0)};
    cuuint32_t estr[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The persistent TMA row pass applies to lines of n1 points when the line
// count fills whole work items.
bool tma_rows_ok(int n1, int64_t lines) { return tma_row_supported(n1) && lines % (4096 / n1) == 0; }

// Which complex64 pass runs the hot modes (kernel variant, lattice, alignment):
// PASS_WARP the warp-synchronous column pass of rk4ip_2d_warp.cu, PASS_TMA the
// persistent passes of rk4ip_2d_tma.cu, PASS_GENERIC the passes of rk4ip_2d.cu.
// Variant 0 takes the TMA row pass and the warp column pass where they apply
// (else the TMA, else the generic column pass); 1 is generic throughout; 2 TMA
// rows with generic columns; 3 the TMA passes for both.
enum { PASS_GENERIC = 0, PASS_TMA = 1, PASS_WARP = 2 };
int row_pass_kind(const xsde_problem *p, int n1, int64_t lines) {
    const int v = p->kernel_variant;
    if (v == 1 || p->grid.basis[p->grid.ndim - 1] != XSDE_BASIS_FOURIER) return PASS_GENERIC;
    return tma_rows_ok(n1, lines) ? PASS_TMA : PASS_GENERIC;
}
int col_pass_kind(const xsde_problem *p, int n0, int64_t n1, int basis0) {
    const int v = p->kernel_variant;
    if (basis0 && p->grid.ndim == 3) return PASS_GENERIC;   // 3D cosine / sine columns: the generic pass
    if (v == 0 && !basis0 && warp_col_supported(n0, n1)) return PASS_WARP;
    if ((v == 0 || v == 3) && tma_col_supported(n0) && n1 % COL_TMA_C == 0) return PASS_TMA;
    return PASS_GENERIC;
}
// tensor maps of fields A and B (rows x cols) for a column pass of that kind;
// a pass whose maps cannot be encoded falls back to the generic kernel
int col_maps(int kind, CUtensorMap *ma, CUtensorMap *mb, void *A, void *B, int64_t rows, int64_t cols, int n0) {
    if (kind == PASS_WARP)
        return encode_field_map_warp(ma, A, rows, cols, n0) && encode_field_map_warp(mb, B, rows, cols, n0)
                   ? PASS_WARP
                   : PASS_GENERIC;
    if (kind == PASS_TMA)
        return encode_field_map(ma, A, rows, cols, n0) && encode_field_map(mb, B, rows, cols, n0) ? PASS_TMA
                                                                                                 : PASS_GENERIC;
    return PASS_GENERIC;
}

// 3D: per exp(L dt/2) application a row pass along dimension 2 (with E2) and
// column passes along dimensions 1 and 0 (E1, E0): the three one-dimensional
// propagators commute.  Sampling splits the run into chunks that end in real
// space; a sample is the row pass's local terms plus a forward transform
// (dimension 2 rows, dimension 1 columns) and the kinetic reduction along
// dimension 0.
// the scratch field B of the 2D/3D pass schedule (grown, never shrunk)
// scratch fields of one 2D / 3D call: B, and C and D with the 2D non-local term
int scratch_fields(const xsde_problem *p) { return p->nonlocal && p->grid.ndim >= 2 ? 3 : 1; }

int ensure_scratch(xsde_problem *p, size_t need, cudaStream_t s) {
    if (p->scratch_bytes >= need) return XSDE_OK;
    if (p->d_scratch) {
        XSDE_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize(scratch)");
        cudaFree(p->d_scratch);
        p->d_scratch = nullptr;
        p->scratch_bytes = 0;
    }
    XSDE_CUDA(cudaMalloc(&p->d_scratch, need), "cudaMalloc(scratch)");
    p->scratch_bytes = need;
    return XSDE_OK;
}

template <typename R>
int run_si_3d(xsde_problem *p, Params2D<R> &qr, Params2D<R> &q1, Params2D<R> &q0, int64_t nsteps, int64_t npaths,
              uint64_t step0, cudaStream_t s);

// RK4IP with the non-local pair potential on a 3D lattice (Example 5's term
// on the 3D trap): the 2D schedule of run_nl_2d, each density convolution
// taking three column passes over C -- dimension 1 forward, dimension 0 with
// the kernel K(k0, k1, k2) (COL_CONV over [n0][n1 n2] columns), dimension 1
// back -- and each propagation two (dimensions 1 and 0).  A sample at step n
// is taken from the real-space field with its V_nl in C, by the row pass's
// NL_FFT and the forward dimension-1 and spectral dimension-0 column passes of
// the local 3D sample.  Generic passes in both precisions.
template <typename R>
int run_nl_3d(xsde_problem *p, Params2D<R> &qr, Params2D<R> &q1, Params2D<R> &q0, int64_t nsteps, uint64_t step0,
              cudaStream_t s) {
    const int S = qr.sm.every;
    const bool sampling = S > 0;
    Params2D<R> c1 = q1;   // the dimension-1 transforms of C (COL_FFT_FWD / COL_FFT_BWD act on B)
    c1.B = q1.C;
    auto row = [&](int op, uint64_t sg, int slot, int last = 0) -> cudaError_t {
        qr.nl_op = op;
        qr.nl_last = last;
        qr.sg = sg;
        qr.sample_slot = slot;
        return timed(p, 9, s, [&] { return launch_row_pass<R>(ROW_NL, qr, s); });
    };
    auto col = [&](Params2D<R> &q, int mode, int slot) -> cudaError_t {
        q.sample_slot = slot;
        const int kind = (mode == COL_CONV || &q == &c1) ? 10 : mode == COL_SPECTRAL ? 8 : 7;
        return timed(p, kind, s, [&] { return launch_col_pass<R>(mode, q, s); });
    };
    auto conv = [&]() -> cudaError_t {
        cudaError_t e = col(c1, COL_FFT_FWD, -1);
        if (e == cudaSuccess) e = col(q0, COL_CONV, -1);
        if (e == cudaSuccess) e = col(c1, COL_FFT_BWD, -1);
        return e;
    };
    auto propagate = [&]() -> cudaError_t {
        cudaError_t e = col(q1, COL_PROPAGATE, -1);
        if (e == cudaSuccess) e = col(q0, COL_PROPAGATE, -1);
        return e;
    };
    // A holds the real-space field of step gs and C its F2 V_nl
    auto sample = [&](int slot, uint64_t gs) -> cudaError_t {
        cudaError_t e = row(NL_FFT, gs, slot);
        if (e == cudaSuccess) e = col(q1, COL_FFT_FWD, -1);
        if (e == cudaSuccess) e = col(q0, COL_SPECTRAL, slot);
        return e;
    };
    if (nsteps > 0) {
        XSDE_CUDA(row(NL_DENSITY, step0, -1), "row pass");
        XSDE_CUDA(conv(), "col pass");
        if (sampling) XSDE_CUDA(sample(0, step0), "sample");
        XSDE_CUDA(row(NL_PROLOGUE, step0, -1), "row pass");
        for (int64_t n = 0; n < nsteps; ++n) {
            const uint64_t sg = step0 + n;
            XSDE_CUDA(propagate(), "col pass");
            XSDE_CUDA(row(NL_S2A, sg, -1), "row pass");
            XSDE_CUDA(conv(), "col pass");
            XSDE_CUDA(row(NL_S2B, sg, -1), "row pass");
            XSDE_CUDA(conv(), "col pass");
            XSDE_CUDA(row(NL_S2C, sg, -1), "row pass");
            XSDE_CUDA(propagate(), "col pass");
            XSDE_CUDA(row(NL_SDA, sg, -1), "row pass");
            XSDE_CUDA(conv(), "col pass");
            const bool last = n + 1 == nsteps;
            XSDE_CUDA(row(NL_SDB, sg, -1, last ? 1 : 0), "row pass");
            if (!last) {
                XSDE_CUDA(conv(), "col pass");
                if (sampling && (n + 1) % S == 0) XSDE_CUDA(sample((int)((n + 1) / S), sg + 1), "sample");
                XSDE_CUDA(row(NL_PROLOGUE, sg + 1, -1), "row pass");
            }
        }
    }
    if (sampling && nsteps % S == 0) {
        XSDE_CUDA(row(NL_DENSITY, step0 + nsteps, -1), "row pass");
        XSDE_CUDA(conv(), "col pass");
        XSDE_CUDA(sample((int)(nsteps / S), step0 + nsteps), "sample");
    }
    return XSDE_OK;
}

template <typename R>
int run_3d(xsde_problem *p, void *psi, int64_t nsteps, int64_t npaths, uint64_t step0, const LocalTerm<R> &lt,
           const Sampling &sm, cudaStream_t s) {
    using V = cx<R>;
    const xsde_grid &g = p->grid;
    int rc_s = ensure_scratch(p, (size_t)scratch_fields(p) * npaths * g.npts * sizeof(V), s);
    if (rc_s != XSDE_OK) return rc_s;
    Params2D<R> base;
    base.A = static_cast<V *>(psi);
    base.B = static_cast<V *>(p->d_scratch);
    base.lt = lt;
    base.sm = sm;
    base.status = p->d_status;
    base.sample_slot = -1;
    base.sg = 0;
    base.ndim = 3;
    Params2D<R> qr = base, q1 = base, q0 = base;
    qr.npaths = npaths;                       // rows: lines along dimension 2
    qr.n0 = g.n[0] * g.n[1];
    qr.n1 = g.n[2];
    qr.nmid = g.n[1];
    qr.tw1 = static_cast<const tw_t<R> *>(p->d_tw[2]);
    qr.E1 = static_cast<const V *>(p->d_E[2]);
    q1.npaths = npaths * g.n[0];              // columns along dimension 1, one slab per (path, i0)
    q1.n0 = g.n[1];
    q1.n1 = g.n[2];
    q1.tw0 = static_cast<const tw_t<R> *>(p->d_tw[1]);
    q1.E0 = static_cast<const V *>(p->d_E[1]);
    q0.npaths = npaths;                       // columns along dimension 0
    q0.n0 = g.n[0];
    q0.n1 = g.n[1] * g.n[2];
    q0.tw0 = static_cast<const tw_t<R> *>(p->d_tw[0]);
    q0.E0 = static_cast<const V *>(p->d_E[0]);
    q0.kinner = g.n[2];
    // cosine / sine dimensions: each pass pairs along its own dimension; the
    // spectral dimension-0 pass weighs the modes of dimensions 1 and 2
    qr.basis1 = g.basis[2];
    qr.B1 = static_cast<const V *>(p->d_B2);
    q1.basis0 = g.basis[1];
    q1.B0 = static_cast<const V *>(p->d_B1);
    q0.basis0 = g.basis[0];
    q0.B0 = static_cast<const V *>(p->d_B);
    q0.basis1 = g.basis[1];
    q0.basis2 = g.basis[2];
    if (p->scheme == XSDE_SCHEME_SEMI_IMPLICIT) {
        if (!p->d_Ef[0] || !p->d_Ef[1] || !p->d_Ef[2]) return fail(XSDE_EINVAL, "semi-implicit 3D step: tables missing");
        return run_si_3d<R>(p, qr, q1, q0, nsteps, npaths, step0, s);
    }
    if (p->nonlocal) {
        for (Params2D<R> *q : {&qr, &q1, &q0}) {
            q->C = base.B + (size_t)npaths * g.npts;
            q->D = q->C + (size_t)npaths * g.npts;
            q->K2 = static_cast<const V *>(p->d_knl);
        }
        return run_nl_3d<R>(p, qr, q1, q0, nsteps, step0, s);
    }
    // complex64: the warp / TMA passes for the hot modes where they apply
    int rk = PASS_GENERIC, ck1 = PASS_GENERIC, ck0 = PASS_GENERIC;
    CUtensorMap map1A, map1B, map0A, map0B;
    if constexpr (std::is_same<R, float>::value) {
        if ((uintptr_t)psi % 16 == 0 && (uintptr_t)p->d_scratch % 16 == 0) {
            rk = row_pass_kind(p, g.n[2], npaths * g.n[0] * g.n[1]);
            // dimension 1: [npaths n0 n1][n2]; dimension 0: [npaths n0][n1 n2]
            ck1 = col_maps(col_pass_kind(p, g.n[1], g.n[2], g.basis[1]), &map1A, &map1B, psi, p->d_scratch,
                           npaths * g.n[0] * g.n[1], g.n[2], g.n[1]);
            ck0 = col_maps(col_pass_kind(p, g.n[0], (int64_t)g.n[1] * g.n[2], g.basis[0]), &map0A, &map0B, psi,
                           p->d_scratch,
                           npaths * g.n[0], (int64_t)g.n[1] * g.n[2], g.n[0]);
            q1.tw0w = static_cast<const tw_t<R> *>(p->d_tw2[1]);
            q0.tw0w = static_cast<const tw_t<R> *>(p->d_tw2[0]);
            qr.tw1p = static_cast<const tw_t<R> *>(p->d_twp);
            if (!qr.tw1p) rk = PASS_GENERIC;
        }
    }
    auto row = [&](int mode, uint64_t sg, int slot) -> cudaError_t {
        qr.sg = sg;
        qr.sample_slot = slot;
        return timed(p, 2 + mode, s, [&] {
            if constexpr (std::is_same<R, float>::value) {
                if (rk == PASS_TMA && (mode == ROW_STAGE2 || mode == ROW_STEADY))
                    return launch_row_pass_tma(mode, qr, p->num_sms, s);
            }
            return launch_row_pass<R>(mode, qr, s);
        });
    };
    auto col = [&](Params2D<R> &q, int mode, int slot) -> cudaError_t {
        q.sample_slot = slot;
        return timed(p, 7 + (mode == COL_SPECTRAL ? 1 : 0), s, [&] {
            if constexpr (std::is_same<R, float>::value) {
                const int kind = &q == &q1 ? ck1 : ck0;
                const CUtensorMap &ma = &q == &q1 ? map1A : map0A, &mb = &q == &q1 ? map1B : map0B;
                if (mode == COL_PROPAGATE && kind == PASS_WARP) return launch_col_pass_warp(q, ma, mb, p->num_sms, s);
                if (mode == COL_PROPAGATE && kind == PASS_TMA) return launch_col_pass_tma(q, ma, mb, p->num_sms, s);
            }
            return launch_col_pass<R>(mode, q, s);
        });
    };
    auto sample = [&](int slot, uint64_t gs) -> int {
        XSDE_CUDA(row(ROW_FFT_ONLY, gs, slot), "row pass");
        XSDE_CUDA(col(q1, COL_FFT_FWD, -1), "col pass");
        XSDE_CUDA(col(q0, COL_SPECTRAL, slot), "col pass");
        return XSDE_OK;
    };
    const int S = sm.every;
    const int64_t chunk = S > 0 ? S : (nsteps > 0 ? nsteps : 1);
    int rc;
    for (int64_t c0 = 0; c0 < nsteps || (S > 0 && c0 == nsteps); c0 += chunk) {
        if (S > 0 && (rc = sample((int)(c0 / S), step0 + c0)) != XSDE_OK) return rc;
        if (c0 == nsteps) break;
        const int64_t len = (c0 + chunk <= nsteps) ? chunk : nsteps - c0;
        XSDE_CUDA(row(ROW_PROLOGUE, step0 + c0, -1), "row pass");
        for (int64_t n = 0; n < len; ++n) {
            const uint64_t sg = step0 + c0 + n;
            XSDE_CUDA(col(q1, COL_PROPAGATE, -1), "col pass");
            XSDE_CUDA(col(q0, COL_PROPAGATE, -1), "col pass");
            XSDE_CUDA(row(ROW_STAGE2, sg, -1), "row pass");
            XSDE_CUDA(col(q1, COL_PROPAGATE, -1), "col pass");
            XSDE_CUDA(col(q0, COL_PROPAGATE, -1), "col pass");
            XSDE_CUDA(row(n + 1 < len ? ROW_STEADY : ROW_EPILOGUE, sg, -1), "row pass");
        }
        if (S > 0 && c0 + len == nsteps && nsteps % S != 0) break;
    }
    return XSDE_OK;
}

// The semi-implicit step on a 2D lattice (XMDS2 Sec. 2.5's semi-implicit
// method in the interaction picture of Sec. 2.6).  One field, A, row-transformed
// between passes (SiOp): a step is one row pass (the three midpoint iterations
// in real space) and one column pass.  Between two steps the half-step factors
// of D (end of step n) and D (start of step n+1) are applied together as the
// whole-step exp(L dt); only where the run samples, or ends, is the state
// brought to a_n itself (half factors, then a multiply-only row pass on the way
// into the next step).  Two passes over one field per step instead of RK4IP's
// four over two.
template <typename R>
int run_si_2d(xsde_problem *p, Params2D<R> &q, int64_t nsteps, uint64_t step0, cudaStream_t s) {
    using V = cx<R>;
    const V *E0h = static_cast<const V *>(p->d_E[0]), *E1h = static_cast<const V *>(p->d_E[1]);
    const V *E0f = static_cast<const V *>(p->d_Ef[0]), *E1f = static_cast<const V *>(p->d_Ef[1]);
    const int S = q.sm.every;
    auto is_sample = [&](int64_t k) { return S > 0 && k % S == 0; };
    auto row = [&](int op, const V *e1, uint64_t sg, int slot) -> cudaError_t {
        q.si_op = op;
        q.E1 = e1;
        q.sg = sg;
        q.sample_slot = slot;
        return timed(p, 4, s, [&] { return launch_row_pass<R>(ROW_SI, q, s); });
    };
    // complex64 columns of 128..512 points take the warp (or TMA) column pass
    // on the one field
    int ck = PASS_GENERIC;
    CUtensorMap mapA, mapA2;
    if constexpr (std::is_same<R, float>::value) {
        if ((uintptr_t)q.A % 16 == 0) {
            int kind = warp_col_supported(q.n0, q.n1) && p->d_tw2[0] ? PASS_WARP
                       : tma_col_supported(q.n0) && q.n1 % COL_TMA_C == 0 ? PASS_TMA
                                                                         : PASS_GENERIC;
            ck = col_maps(kind, &mapA, &mapA2, q.A, q.A, q.npaths * q.n0, q.n1, q.n0);
        }
        q.tw0w = static_cast<const tw_t<R> *>(p->d_tw2[0]);
    }
    auto col = [&](const V *e0) -> cudaError_t {
        q.E0 = e0;
        q.sample_slot = -1;
        return timed(p, 7, s, [&] {
            if constexpr (std::is_same<R, float>::value)
                if (ck != PASS_GENERIC) {
                    Params2D<float> t = q;
                    t.single_field = 1;
                    return ck == PASS_WARP ? launch_col_pass_warp(t, mapA, mapA, p->num_sms, s)
                                           : launch_col_pass_tma(t, mapA, mapA, p->num_sms, s);
                }
            return launch_col_pass<R>(COL_SINGLE, q, s);
        });
    };
    auto kinetic = [&](int slot) -> cudaError_t {   // the spectral energy of the state F1 a / n1
        Params2D<R> k = q;
        k.B = q.A;
        k.sample_slot = slot;
        k.spec_scale = (double)q.n1 * (double)q.n1;
        return timed(p, 8, s, [&] { return launch_col_pass<R>(COL_SPECTRAL, k, s); });
    };
    XSDE_CUDA(row(SI_ENTER, E1h, step0, -1), "row pass");   // state: F1 a_0 / n1
    bool at_a = true;                                        // state holds a_k (not D a_k)
    for (int64_t k = 0; k <= nsteps; ++k) {
        const int slot = is_sample(k) ? (int)(k / S) : -1;
        if (k == nsteps) {
            if (slot >= 0) XSDE_CUDA(kinetic(slot), "col pass");
            XSDE_CUDA(row(SI_EXIT, E1h, step0 + k, slot), "row pass");
            break;
        }
        if (at_a) {   // into step k: F1 a_k / n1 -> F1 D a_k / n1
            if (slot >= 0) XSDE_CUDA(kinetic(slot), "col pass");
            XSDE_CUDA(row(SI_MUL, E1h, step0 + k, slot), "row pass");
            XSDE_CUDA(col(E0h), "col pass");
        }
        // step k; then either stop at a_{k+1} or go straight on into step k+1
        at_a = k + 1 == nsteps || is_sample(k + 1);
        XSDE_CUDA(row(SI_STEP, at_a ? E1h : E1f, step0 + k, -1), "row pass");
        XSDE_CUDA(col(at_a ? E0h : E0f), "col pass");
    }
    return XSDE_OK;
}

// The same schedule on a 3D lattice: the row pass runs along dimension 2, the
// column passes along dimensions 1 and 0 (each on the one field); the state
// between passes is F2 u / n2.  The spectral energy needs F1 of the state, taken
// on a copy in the scratch field.
template <typename R>
int run_si_3d(xsde_problem *p, Params2D<R> &qr, Params2D<R> &q1, Params2D<R> &q0, int64_t nsteps, int64_t npaths,
              uint64_t step0, cudaStream_t s) {
    using V = cx<R>;
    const V *Eh[3], *Ef[3];
    for (int d = 0; d < 3; ++d) {
        Eh[d] = static_cast<const V *>(p->d_E[d]);
        Ef[d] = static_cast<const V *>(p->d_Ef[d]);
    }
    const int S = qr.sm.every;
    auto is_sample = [&](int64_t k) { return S > 0 && k % S == 0; };
    auto row = [&](int op, bool whole, uint64_t sg, int slot) -> cudaError_t {
        qr.si_op = op;
        qr.E1 = whole ? Ef[2] : Eh[2];
        qr.sg = sg;
        qr.sample_slot = slot;
        return timed(p, 4, s, [&] { return launch_row_pass<R>(ROW_SI, qr, s); });
    };
    auto cols = [&](bool whole) -> cudaError_t {
        q1.E0 = whole ? Ef[1] : Eh[1];
        q0.E0 = whole ? Ef[0] : Eh[0];
        q1.sample_slot = q0.sample_slot = -1;
        cudaError_t e = timed(p, 7, s, [&] { return launch_col_pass<R>(COL_SINGLE, q1, s); });
        if (e != cudaSuccess) return e;
        return timed(p, 7, s, [&] { return launch_col_pass<R>(COL_SINGLE, q0, s); });
    };
    auto kinetic = [&](int slot) -> cudaError_t {
        const size_t bytes = (size_t)npaths * p->grid.npts * sizeof(V);
        cudaError_t e = cudaMemcpyAsync(q1.B, q1.A, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        e = timed(p, 8, s, [&] { return launch_col_pass<R>(COL_FFT_FWD, q1, s); });
        if (e != cudaSuccess) return e;
        Params2D<R> k = q0;
        k.sample_slot = slot;
        k.spec_scale = (double)qr.n1 * (double)qr.n1;
        return timed(p, 8, s, [&] { return launch_col_pass<R>(COL_SPECTRAL, k, s); });
    };
    XSDE_CUDA(row(SI_ENTER, false, step0, -1), "row pass");
    bool at_a = true;
    for (int64_t k = 0; k <= nsteps; ++k) {
        const int slot = is_sample(k) ? (int)(k / S) : -1;
        if (k == nsteps) {
            if (slot >= 0) XSDE_CUDA(kinetic(slot), "col pass");
            XSDE_CUDA(row(SI_EXIT, false, step0 + k, slot), "row pass");
            break;
        }
        if (at_a) {
            if (slot >= 0) XSDE_CUDA(kinetic(slot), "col pass");
            XSDE_CUDA(row(SI_MUL, false, step0 + k, slot), "row pass");
            XSDE_CUDA(cols(false), "col pass");
        }
        at_a = k + 1 == nsteps || is_sample(k + 1);
        XSDE_CUDA(row(SI_STEP, !at_a, step0 + k, -1), "row pass");
        XSDE_CUDA(cols(!at_a), "col pass");
    }
    return XSDE_OK;
}

// RK4IP with the non-local pair potential (Example 5) on a 2D lattice, generic
// passes.  Every evaluation of N reads the V_nl of its own argument, so each is
// preceded by a density convolution (NlOp): a row pass forms C = F1 |u|^2, a
// column pass COL_CONV takes it to F1 V_nl, the next row pass uses it.  A step:
//   col(propagate) S2A conv S2B conv S2C col(propagate) SDA conv SDB [conv PROLOGUE]
// i.e. 6 row passes, 2 propagating and 4 convolving column passes (the
// prologue of the next step is the tail of this one).
template <typename R>
int run_nl_2d(xsde_problem *p, Params2D<R> &q, int64_t nsteps, uint64_t step0, cudaStream_t s) {
    const int S = q.sm.every;
    const bool sampling = S > 0;
    auto row = [&](int op, uint64_t sg, int slot, int last = 0) -> cudaError_t {
        q.nl_op = op;
        q.nl_last = last;
        q.sg = sg;
        q.sample_slot = slot;
        return timed(p, 9, s, [&] { return launch_row_pass<R>(ROW_NL, q, s); });
    };
    auto col = [&](int mode, int slot) -> cudaError_t {
        q.sample_slot = slot;
        return timed(p, mode == COL_CONV ? 10 : 7, s, [&] { return launch_col_pass<R>(mode, q, s); });
    };
    if (nsteps > 0) {
        XSDE_CUDA(row(NL_DENSITY, step0, -1), "row pass");
        XSDE_CUDA(col(COL_CONV, -1), "col pass");
        XSDE_CUDA(row(NL_PROLOGUE, step0, sampling ? 0 : -1), "row pass");
        for (int64_t n = 0; n < nsteps; ++n) {
            const uint64_t sg = step0 + n;
            XSDE_CUDA(col(COL_PROPAGATE, (sampling && n % S == 0) ? (int)(n / S) : -1), "col pass");
            XSDE_CUDA(row(NL_S2A, sg, -1), "row pass");
            XSDE_CUDA(col(COL_CONV, -1), "col pass");
            XSDE_CUDA(row(NL_S2B, sg, -1), "row pass");
            XSDE_CUDA(col(COL_CONV, -1), "col pass");
            XSDE_CUDA(row(NL_S2C, sg, -1), "row pass");
            XSDE_CUDA(col(COL_PROPAGATE, -1), "col pass");
            XSDE_CUDA(row(NL_SDA, sg, -1), "row pass");
            XSDE_CUDA(col(COL_CONV, -1), "col pass");
            const bool last = n + 1 == nsteps;
            XSDE_CUDA(row(NL_SDB, sg, -1, last ? 1 : 0), "row pass");
            if (!last) {
                XSDE_CUDA(col(COL_CONV, -1), "col pass");
                const int slot = (sampling && (n + 1) % S == 0) ? (int)((n + 1) / S) : -1;
                XSDE_CUDA(row(NL_PROLOGUE, sg + 1, slot), "row pass");
            }
        }
    }
    if (sampling && nsteps % S == 0) {
        const int slot = (int)(nsteps / S);
        XSDE_CUDA(row(NL_DENSITY, step0 + nsteps, -1), "row pass");
        XSDE_CUDA(col(COL_CONV, -1), "col pass");
        XSDE_CUDA(row(NL_FFT, step0 + nsteps, slot), "row pass");
        XSDE_CUDA(col(COL_SPECTRAL, slot), "col pass");
    }
    return XSDE_OK;
}

template <typename R>
int run_integrate(xsde_problem *p, void *psi, double dt, int64_t nsteps, int64_t npaths, int64_t path_offset,
                  uint64_t step0, cudaStream_t s) {
    using V = cx<R>;
    int rc = ensure_tables<V>(p, dt, s);
    if (rc != XSDE_OK) return rc;
    LocalTerm<R> lt;
    Sampling sm;
    fill_terms<R>(p, dt, npaths, path_offset, lt, sm);
    const xsde_grid &g = p->grid;
    const bool sampling = sm.every > 0;
    sm.nsamp = sampling ? nsteps / sm.every + 1 : 0;
    if (sampling) {
        const int64_t nsamp = nsteps / sm.every + 1;
        if (sm.per_path && (sm.which & (MOM_NORM | MOM_ENERGY)))
            XSDE_CUDA(cudaMemsetAsync(sm.per_path, 0, (size_t)nsamp * npaths * 2 * sizeof(double), s), "memset");
        if (sm.per_point && (sm.which & (MOM_MOD2 | MOM_MOD4)))
            XSDE_CUDA(cudaMemsetAsync(sm.per_point, 0, (size_t)nsamp * g.npts * 2 * sizeof(double), s), "memset");
    }

    if (g.ndim == 0) {
        Params0D<R> q;
        q.psi = static_cast<V *>(psi);
        q.npaths = npaths;
        q.nsteps = nsteps;
        q.step0 = step0;
        const std::complex<double> eh = std::exp(std::complex<double>(p->L.c0_re, p->L.c0_im) * (0.5 * dt));
        q.Ehalf.x = (R)eh.real();
        q.Ehalf.y = (R)eh.imag();
        q.lt = lt;
        q.sm = sm;
        q.status = p->d_status;
        q.scheme = p->scheme;
        XSDE_CUDA(timed(p, 0, s, [&] { return launch_rk4ip_0d<R>(q, s); }), "rk4ip_0d launch");
        return XSDE_OK;
    }
    if (g.ndim == 1) {
        Params1D<R> q;
        q.psi = static_cast<V *>(psi);
        q.npaths = npaths;
        q.nsteps = nsteps;
        q.step0 = step0;
        q.Etab = static_cast<const V *>(p->d_E[0]);
        const bool shape0 = p->scheme != XSDE_SCHEME_RK4IP || p->nonlocal || g.basis[0] != XSDE_BASIS_FOURIER;
        const int elems = shape0 ? 8 : rk4ip_1d_elems(p->kernel_variant);
        q.tw = static_cast<const tw_t<R> *>(elems == 8 ? p->d_tw[0] : p->d_tw1d[elems == 4 ? 0 : 1]);
        q.lt = lt;
        q.sm = sm;
        q.status = p->d_status;
        q.scheme = p->scheme;
        q.knl = p->nonlocal ? static_cast<const V *>(p->d_knl) : nullptr;
        q.basis = g.basis[0];
        q.Btab = static_cast<const V *>(p->d_B);
        XSDE_CUDA(timed(p, 1, s, [&] { return launch_rk4ip_1d<R>(g.n[0], p->kernel_variant, q, s); }),
                  "rk4ip_1d launch");
        return XSDE_OK;
    }
    if (g.ndim == 3) return run_3d<R>(p, psi, nsteps, npaths, step0, lt, sm, s);
    // 2D: scratch field B (same shape as psi); C and D with the non-local term
    int rc_s = ensure_scratch(p, (size_t)scratch_fields(p) * npaths * g.npts * sizeof(V), s);
    if (rc_s != XSDE_OK) return rc_s;
    Params2D<R> q;
    q.A = static_cast<V *>(psi);
    q.B = static_cast<V *>(p->d_scratch);
    q.npaths = npaths;
    q.n0 = g.n[0];
    q.n1 = g.n[1];
    q.tw0 = static_cast<const tw_t<R> *>(p->d_tw[0]);
    q.tw1 = static_cast<const tw_t<R> *>(p->d_tw[1]);
    q.E0 = static_cast<const V *>(p->d_E[0]);
    q.E1 = static_cast<const V *>(p->d_E[1]);
    q.lt = lt;
    q.sm = sm;
    q.status = p->d_status;
    q.basis0 = g.basis[0];
    q.B0 = static_cast<const V *>(p->d_B);
    q.basis1 = g.basis[1];
    q.B1 = static_cast<const V *>(p->d_B1);
    const int S = sm.every;
    if (p->scheme == XSDE_SCHEME_SEMI_IMPLICIT) {
        if (!p->d_Ef[0] || !p->d_Ef[1]) return fail(XSDE_EINVAL, "semi-implicit 2D step: tables missing");
        return run_si_2d<R>(p, q, nsteps, step0, s);
    }
    if (p->nonlocal) {
        q.C = q.B + (size_t)npaths * g.npts;
        q.D = q.C + (size_t)npaths * g.npts;
        q.K2 = static_cast<const V *>(p->d_knl);
        return run_nl_2d<R>(p, q, nsteps, step0, s);
    }
    // complex64 lattices the warp / TMA passes cover take the hot modes there
    int rk = PASS_GENERIC, ck = PASS_GENERIC;
    CUtensorMap mapA, mapB;
    if constexpr (std::is_same<R, float>::value) {
        if ((uintptr_t)psi % 16 == 0 && (uintptr_t)p->d_scratch % 16 == 0) {
            rk = row_pass_kind(p, g.n[1], npaths * g.n[0]);
            ck = col_maps(col_pass_kind(p, g.n[0], g.n[1], g.basis[0]), &mapA, &mapB, psi, p->d_scratch,
                          npaths * g.n[0], g.n[1], g.n[0]);
        }
        q.tw0w = static_cast<const tw_t<R> *>(p->d_tw2[0]);
        q.tw1p = static_cast<const tw_t<R> *>(p->d_twp);
        if (!q.tw1p) rk = PASS_GENERIC;
    }
    auto row = [&](int mode, uint64_t sg, int slot) -> cudaError_t {
        q.sg = sg;
        q.sample_slot = slot;
        return timed(p, 2 + mode, s, [&] {
            if constexpr (std::is_same<R, float>::value) {
                if (rk == PASS_TMA && (mode == ROW_STAGE2 || mode == ROW_STEADY))
                    return launch_row_pass_tma(mode, q, p->num_sms, s);
            }
            return launch_row_pass<R>(mode, q, s);
        });
    };
    auto col = [&](int mode, int slot) -> cudaError_t {
        q.sample_slot = slot;
        return timed(p, 7 + mode, s, [&] {
            if constexpr (std::is_same<R, float>::value) {
                if (ck == PASS_WARP && mode == COL_PROPAGATE) return launch_col_pass_warp(q, mapA, mapB, p->num_sms, s);
                if (ck == PASS_TMA && mode == COL_PROPAGATE) return launch_col_pass_tma(q, mapA, mapB, p->num_sms, s);
            }
            return launch_col_pass<R>(mode, q, s);
        });
    };
    if (g.basis[1] != XSDE_BASIS_FOURIER) {
        // a cosine / sine dimension 1: the fused sample of the column pass needs
        // the Fourier row spectrum, so samples are taken from the real-space
        // field between chunks of steps (the 3D schedule): the row pass's
        // cosine / sine spectrum and a spectral column pass
        const int64_t chunk = S > 0 ? S : (nsteps > 0 ? nsteps : 1);
        for (int64_t c0 = 0; c0 < nsteps || (S > 0 && c0 == nsteps); c0 += chunk) {
            if (S > 0) {
                XSDE_CUDA(row(ROW_FFT_ONLY, step0 + c0, (int)(c0 / S)), "row pass");
                XSDE_CUDA(col(COL_SPECTRAL, (int)(c0 / S)), "col pass");
            }
            if (c0 == nsteps) break;
            const int64_t len = (c0 + chunk <= nsteps) ? chunk : nsteps - c0;
            XSDE_CUDA(row(ROW_PROLOGUE, step0 + c0, -1), "row pass");
            for (int64_t n = 0; n < len; ++n) {
                const uint64_t sg = step0 + c0 + n;
                XSDE_CUDA(col(COL_PROPAGATE, -1), "col pass");
                XSDE_CUDA(row(ROW_STAGE2, sg, -1), "row pass");
                XSDE_CUDA(col(COL_PROPAGATE, -1), "col pass");
                XSDE_CUDA(row(n + 1 < len ? ROW_STEADY : ROW_EPILOGUE, sg, -1), "row pass");
            }
            if (S > 0 && c0 + len == nsteps && nsteps % S != 0) break;
        }
        return XSDE_OK;
    }
    if (nsteps > 0) {
        XSDE_CUDA(row(ROW_PROLOGUE, step0, sampling ? 0 : -1), "row pass");
        for (int64_t n = 0; n < nsteps; ++n) {
            const uint64_t sg = step0 + n;
            XSDE_CUDA(col(COL_PROPAGATE, (sampling && n % S == 0) ? (int)(n / S) : -1), "col pass");
            XSDE_CUDA(row(ROW_STAGE2, sg, -1), "row pass");
            XSDE_CUDA(col(COL_PROPAGATE, -1), "col pass");
            if (n + 1 < nsteps) {
                const int slot = (sampling && (n + 1) % S == 0) ? (int)((n + 1) / S) : -1;
                XSDE_CUDA(row(ROW_STEADY, sg, slot), "row pass");
            } else {
                XSDE_CUDA(row(ROW_EPILOGUE, sg, -1), "row pass");
            }
        }
    }
    if (sampling && nsteps % S == 0) {
        const int slot = (int)(nsteps / S);
        XSDE_CUDA(row(ROW_FFT_ONLY, step0 + nsteps, slot), "row pass");
        XSDE_CUDA(col(COL_SPECTRAL, slot), "col pass");
    }
    return XSDE_OK;
}

bool same_lattice(const xsde_grid &a, const xsde_grid &b) {
    if (a.ndim != b.ndim) return false;
    for (int d = 0; d < a.ndim; ++d)
        if (a.n[d] != b.n[d] || a.xmin[d] != b.xmin[d] || a.xmax[d] != b.xmax[d] || a.basis[d] != b.basis[d])
            return false;
    return true;
}

// Argument checks shared by the integrating entry points.
int check_integrate(const char *who, xsde_problem *p, const xsde_vector *psi, double dt, int64_t nsteps,
                    int64_t npaths, int64_t path_offset, uint64_t step_offset) {
    if (!p || !psi) return fail(XSDE_EINVAL, "%s: NULL problem or field", who);
    if (!p->have_ops) return fail(XSDE_EINVAL, "%s: operators not set", who);
    if (psi->dtype != p->dtype) return fail(XSDE_EINVAL, "%s: field dtype differs from the problem's", who);
    if (!same_lattice(psi->grid, p->grid)) return fail(XSDE_EINVAL, "%s: field lattice differs", who);
    if (npaths != psi->npaths)
        return fail(XSDE_EINVAL, "%s: npaths %lld != field npaths %lld", who, (long long)npaths,
                    (long long)psi->npaths);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(XSDE_EINVAL, "%s: dt must be positive and finite", who);
    if (nsteps < 0) return fail(XSDE_EINVAL, "%s: nsteps < 0", who);
    if (path_offset < 0 || path_offset + npaths > (int64_t)UINT32_MAX + 1)
        return fail(XSDE_EINVAL, "%s: global path indices exceed 32 bits", who);
    if ((step_offset + (uint64_t)nsteps + 1) * (uint64_t)p->noise_substeps > (uint64_t)UINT32_MAX)
        return fail(XSDE_EINVAL, "%s: global step indices exceed 32 bits", who);
    if (p->N.pot_kind == XSDE_POT_TABLE && p->N.V_nt > 1 && step_offset + (uint64_t)nsteps > (uint64_t)p->N.V_nt)
        return fail(XSDE_EINVAL, "%s: potential table has %lld rows, steps up to %llu needed", who,
                    (long long)p->N.V_nt, (unsigned long long)(step_offset + nsteps));
    if (p->grid.ndim == 3 && npaths * p->grid.n[0] > 65535)
        return fail(XSDE_EUNSUPPORTED, "%s: at most 65535 paths x n0 slabs per call on a 3D lattice", who);
    if (p->grid.ndim == 2 && npaths > 65535)
        return fail(XSDE_EUNSUPPORTED, "%s: at most 65535 paths per call on a 2D lattice", who);
    if (p->samp.every > 0 && nsteps / p->samp.every + 1 > (int64_t)INT32_MAX)
        return fail(XSDE_EINVAL, "%s: too many samples", who);
    if (p->nonlocal && p->scheme != XSDE_SCHEME_RK4IP)
        return fail(XSDE_EUNSUPPORTED, "%s: the non-local term runs with RK4IP only", who);
    if (any_basis(p->grid)) {
        const xsde_grid &g = p->grid;
        if (g.ndim >= 2 && p->scheme != XSDE_SCHEME_RK4IP)
            return fail(XSDE_EUNSUPPORTED, "%s: the semi-implicit scheme on 2D / 3D Fourier lattices only", who);
    }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) return fail(XSDE_EINVAL, "%s: current device %d is not the problem's %d", who, dev, p->device);
    return XSDE_OK;
}

int integrate_on(xsde_problem *p, void *psi, double dt, int64_t nsteps, int64_t npaths, int64_t path_offset,
                 uint64_t step_offset, cudaStream_t s) {
    return p->dtype == XSDE_C64 ? run_integrate<float>(p, psi, dt, nsteps, npaths, path_offset, step_offset, s)
                                : run_integrate<double>(p, psi, dt, nsteps, npaths, path_offset, step_offset, s);
}

// Number of kernel variants the lattice offers (xsde_set_kernel_variant).
int variants_for(const xsde_problem *p) {
    switch (p->grid.ndim) {
        // the semi-implicit step, the non-local term and cosine / sine lattices
        // have one launch shape
        case 1:
            return p->scheme != XSDE_SCHEME_RK4IP || p->nonlocal || p->grid.basis[0] != XSDE_BASIS_FOURIER
                       ? 1
                       : rk4ip_1d_variants();
        case 2:
        case 3:   // the semi-implicit step and the 2D non-local term: one shape
            return p->scheme != XSDE_SCHEME_RK4IP || p->nonlocal ? 1 : 4;
        default: return 1;
    }
}

}  // namespace

extern "C" {

const char *xsde_last_error(void) { return g_err.c_str(); }
const char *xsde_version(void) { return "xsde 0.1 (sm_103a)"; }

int xsde_grid_create(int ndim, const int32_t *npts, const double *xmin, const double *xmax, xsde_grid **out) {
    if (!out) return fail(XSDE_EINVAL, "xsde_grid_create: out is NULL");
    *out = nullptr;
    if (ndim < 0 || ndim > 3) return fail(XSDE_EINVAL, "xsde_grid_create: ndim %d not in 0..3", ndim);
    if (ndim > 0 && (!npts || !xmin || !xmax)) return fail(XSDE_EINVAL, "xsde_grid_create: NULL array");
    xsde_grid g{};
    g.ndim = ndim;
    g.npts = 1;
    for (int d = 0; d < ndim; ++d) {
        if (!pow2_in_range(npts[d]))
            return fail(XSDE_EINVAL, "xsde_grid_create: npts[%d] = %d is not a power of two in [16, 2048]", d, npts[d]);
        if (!(xmin[d] < xmax[d]) || !std::isfinite(xmin[d]) || !std::isfinite(xmax[d]))
            return fail(XSDE_EINVAL, "xsde_grid_create: domain [%g, %g) of dimension %d is empty", xmin[d], xmax[d], d);
        g.n[d] = npts[d];
        g.xmin[d] = xmin[d];
        g.xmax[d] = xmax[d];
        g.npts *= npts[d];
    }
    xsde_grid *p = new (std::nothrow) xsde_grid(g);
    if (!p) return fail(XSDE_ENOMEM, "xsde_grid_create: out of host memory");
    *out = p;
    return XSDE_OK;
}

void xsde_grid_destroy(xsde_grid *grid) { delete grid; }

int xsde_grid_set_basis(xsde_grid *grid, const int32_t *basis) {
    if (!grid) return fail(XSDE_EINVAL, "xsde_grid_set_basis: grid is NULL");
    if (grid->ndim > 0 && !basis) return fail(XSDE_EINVAL, "xsde_grid_set_basis: basis is NULL");
    for (int d = 0; d < grid->ndim; ++d)
        if (basis[d] < XSDE_BASIS_FOURIER || basis[d] > XSDE_BASIS_SIN)
            return fail(XSDE_EINVAL, "xsde_grid_set_basis: basis[%d] = %d", d, basis[d]);
    for (int d = 0; d < grid->ndim; ++d) grid->basis[d] = basis[d];
    return XSDE_OK;
}

int64_t xsde_grid_points(const xsde_grid *grid) { return grid ? grid->npts : 0; }

static int vector_check(const xsde_grid *grid, xsde_dtype dtype, int ncomp, int64_t npaths, xsde_vector **out) {
    if (!out) return fail(XSDE_EINVAL, "vector: out is NULL");
    *out = nullptr;
    if (!grid) return fail(XSDE_EINVAL, "vector: grid is NULL");
    if (dtype != XSDE_C64 && dtype != XSDE_C128) return fail(XSDE_EINVAL, "vector: unknown dtype %d", (int)dtype);
    if (ncomp != 1) return fail(XSDE_EUNSUPPORTED, "vector: ncomp = %d (only 1 component is supported)", ncomp);
    if (npaths < 1 || npaths > (int64_t)UINT32_MAX) return fail(XSDE_EINVAL, "vector: npaths = %lld", (long long)npaths);
    return XSDE_OK;
}

int xsde_vector_alloc(const xsde_grid *grid, xsde_dtype dtype, int ncomp, int64_t npaths, xsde_vector **out) {
    int rc = vector_check(grid, dtype, ncomp, npaths, out);
    if (rc != XSDE_OK) return rc;
    const size_t bytes = (size_t)npaths * grid->npts * elem_bytes(dtype);
    void *d = nullptr;
    XSDE_CUDA(cudaMalloc(&d, bytes), "xsde_vector_alloc");
    cudaError_t e = cudaMemset(d, 0, bytes);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "xsde_vector_alloc: memset");
    }
    *out = new xsde_vector{*grid, dtype, ncomp, npaths, d, true};
    return XSDE_OK;
}

int xsde_vector_wrap(const xsde_grid *grid, xsde_dtype dtype, int ncomp, int64_t npaths, void *dev_ptr,
                     xsde_vector **out) {
    int rc = vector_check(grid, dtype, ncomp, npaths, out);
    if (rc != XSDE_OK) return rc;
    if (!dev_ptr) return fail(XSDE_EINVAL, "xsde_vector_wrap: dev_ptr is NULL");
    if ((uintptr_t)dev_ptr % elem_bytes(dtype))
        return fail(XSDE_EINVAL, "xsde_vector_wrap: dev_ptr not aligned to %zu bytes", elem_bytes(dtype));
    *out = new xsde_vector{*grid, dtype, ncomp, npaths, dev_ptr, false};
    return XSDE_OK;
}

void *xsde_vector_data(const xsde_vector *vec) { return vec ? vec->data : nullptr; }

void xsde_vector_free(xsde_vector *vec) {
    if (!vec) return;
    if (vec->owned) cudaFree(vec->data);
    delete vec;
}

int xsde_noise_alloc(const xsde_grid *grid, xsde_noise_kind kind, uint64_t seed, xsde_noise **out) {
    if (!out) return fail(XSDE_EINVAL, "xsde_noise_alloc: out is NULL");
    *out = nullptr;
    if (!grid) return fail(XSDE_EINVAL, "xsde_noise_alloc: grid is NULL");
    if (kind != XSDE_NOISE_WIENER_REAL && kind != XSDE_NOISE_WIENER_COMPLEX)
        return fail(XSDE_EINVAL, "xsde_noise_alloc: unknown kind %d", (int)kind);
    *out = new xsde_noise{kind, seed};
    return XSDE_OK;
}

void xsde_noise_free(xsde_noise *noise) { delete noise; }

int xsde_problem_create(const xsde_grid *grid, xsde_dtype dtype, xsde_problem **out) {
    if (!out) return fail(XSDE_EINVAL, "xsde_problem_create: out is NULL");
    *out = nullptr;
    if (!grid) return fail(XSDE_EINVAL, "xsde_problem_create: grid is NULL");
    if (dtype != XSDE_C64 && dtype != XSDE_C128) return fail(XSDE_EINVAL, "xsde_problem_create: unknown dtype");
    xsde_problem *p = new (std::nothrow) xsde_problem();
    if (!p) return fail(XSDE_ENOMEM, "xsde_problem_create: out of host memory");
    p->grid = *grid;
    p->dtype = dtype;
    cudaGetDevice(&p->device);
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (p->num_sms < 1) p->num_sms = 1;
    cudaError_t e = cudaMalloc(&p->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "xsde_problem_create");
    }
    *out = p;
    return XSDE_OK;
}

void xsde_problem_destroy(xsde_problem *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    for (auto &m : p->marks) {
        cudaEventDestroy(m.start);
        cudaEventDestroy(m.stop);
    }
    for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
    for (int d = 0; d < 3; ++d) {
        cudaFree(p->d_tw[d]);
        cudaFree(p->d_E[d]);
    }
    cudaFree(p->d_tw1d[0]);
    cudaFree(p->d_tw1d[1]);
    for (int d = 0; d < 3; ++d) cudaFree(p->d_tw2[d]);
    cudaFree(p->d_twp);
    cudaFree(p->d_knl);
    cudaFree(p->d_B);
    cudaFree(p->d_B1);
    cudaFree(p->d_B2);
    for (int d = 0; d < 3; ++d) cudaFree(p->d_Ef[d]);
    cudaFree(p->d_scratch);
    cudaFree(p->d_adj);
    cudaFree(p->d_status);
    cudaFree(p->d_plain);
    cudaFree(p->d_plain_E);
    cudaFree(p->d_hostfield);
    plain_plan_destroy(p->plain);
    delete p;
}

int xsde_set_operators(xsde_problem *p, const xsde_linear_op *L, const xsde_nonlinear_op *N) {
    if (!p || !L || !N) return fail(XSDE_EINVAL, "xsde_set_operators: NULL argument");
    const double vals[] = {L->c0_re, L->c0_im, L->c2_re, L->c2_im, N->g, N->amplitude,
                           N->omega[0], N->omega[1], N->omega[2]};
    for (double v : vals)
        if (!std::isfinite(v)) return fail(XSDE_EINVAL, "xsde_set_operators: non-finite coefficient");
    if (N->pot_kind < XSDE_POT_NONE || N->pot_kind > XSDE_POT_TABLE)
        return fail(XSDE_EINVAL, "xsde_set_operators: unknown pot_kind %d", N->pot_kind);
    if (N->pot_kind == XSDE_POT_TABLE && (!N->V || N->V_nt < 1))
        return fail(XSDE_EINVAL, "xsde_set_operators: potential table needs V != NULL and V_nt >= 1");
    if (N->coupling != XSDE_COUPLE_ADDITIVE && N->coupling != XSDE_COUPLE_MULTIPLICATIVE)
        return fail(XSDE_EINVAL, "xsde_set_operators: unknown coupling %d", N->coupling);
    if (N->noise && N->coupling == XSDE_COUPLE_MULTIPLICATIVE && N->noise->kind != XSDE_NOISE_WIENER_REAL)
        return fail(XSDE_EINVAL, "xsde_set_operators: multiplicative coupling needs real noise");
    p->L = *L;
    p->N = *N;
    p->noise = N->noise ? *N->noise : xsde_noise{XSDE_NOISE_NONE, 0};
    p->N.noise = nullptr;
    p->have_ops = true;
    p->table_dt = -1.0;
    ++p->generation;
    return XSDE_OK;
}

int xsde_moments(xsde_problem *p, const xsde_sampling *spec, double *per_path, double *per_point) {
    if (!p) return fail(XSDE_EINVAL, "xsde_moments: problem is NULL");
    if (!spec || spec->every == 0) {
        p->samp = xsde_sampling{0, 0};
        p->per_path = p->per_point = nullptr;
        ++p->generation;
        return XSDE_OK;
    }
    if (spec->every < 0) return fail(XSDE_EINVAL, "xsde_moments: every = %d", spec->every);
    if (spec->which & ~(XSDE_MOM_NORM | XSDE_MOM_ENERGY | XSDE_MOM_MOD2 | XSDE_MOM_MOD4))
        return fail(XSDE_EINVAL, "xsde_moments: unknown moment bits 0x%x", spec->which);
    if ((spec->which & (XSDE_MOM_NORM | XSDE_MOM_ENERGY)) && !per_path)
        return fail(XSDE_EINVAL, "xsde_moments: NORM/ENERGY requested without per_path buffer");
    if ((spec->which & (XSDE_MOM_MOD2 | XSDE_MOM_MOD4)) && !per_point)
        return fail(XSDE_EINVAL, "xsde_moments: MOD2/MOD4 requested without per_point buffer");
    p->samp = *spec;
    p->per_path = per_path;
    p->per_point = per_point;
    ++p->generation;
    return XSDE_OK;
}

int xsde_integrate(xsde_problem *p, xsde_vector *psi, double dt, int64_t nsteps, int64_t npaths,
                   int64_t path_offset, uint64_t step_offset, void *stream) {
    const int rc = check_integrate("xsde_integrate", p, psi, dt, nsteps, npaths, path_offset, step_offset);
    if (rc != XSDE_OK) return rc;
    return integrate_on(p, psi->data, dt, nsteps, npaths, path_offset, step_offset, static_cast<cudaStream_t>(stream));
}

int xsde_integrate_host(xsde_problem *p, const void *psi_in, void *psi_out, int64_t npaths, double dt,
                        int64_t nsteps, int64_t path_offset, uint64_t step_offset, void *stream) {
    const char *who = "xsde_integrate_host";
    if (!p || !psi_in || !psi_out) return fail(XSDE_EINVAL, "%s: NULL problem or host field", who);
    if (npaths < 1) return fail(XSDE_EINVAL, "%s: npaths must be >= 1", who);
    const size_t bytes = (size_t)npaths * p->grid.npts * elem_bytes(p->dtype);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->hostfield_bytes < bytes) {
        if (p->d_hostfield) {
            XSDE_CUDA(cudaStreamSynchronize(s), "xsde_integrate_host: field");
            cudaFree(p->d_hostfield);
            p->d_hostfield = nullptr;
            p->hostfield_bytes = 0;
        }
        XSDE_CUDA(cudaMalloc(&p->d_hostfield, bytes), "xsde_integrate_host: field");
        p->hostfield_bytes = bytes;
    }
    xsde_vector dev{p->grid, p->dtype, 1, npaths, p->d_hostfield, false};
    int rc = check_integrate(who, p, &dev, dt, nsteps, npaths, path_offset, step_offset);
    if (rc != XSDE_OK) return rc;
    XSDE_CUDA(cudaMemcpyAsync(p->d_hostfield, psi_in, bytes, cudaMemcpyHostToDevice, s), "xsde_integrate_host: copy in");
    rc = integrate_on(p, p->d_hostfield, dt, nsteps, npaths, path_offset, step_offset, s);
    if (rc != XSDE_OK) return rc;
    XSDE_CUDA(cudaMemcpyAsync(psi_out, p->d_hostfield, bytes, cudaMemcpyDeviceToHost, s), "xsde_integrate_host: copy out");
    return XSDE_OK;
}

int xsde_set_kernel_variant(xsde_problem *p, int variant) {
    if (!p) return fail(XSDE_EINVAL, "xsde_set_kernel_variant: problem is NULL");
    if (variant < 0 || variant >= variants_for(p))
        return fail(XSDE_EINVAL, "xsde_set_kernel_variant: variant %d (the lattice has %d)", variant, variants_for(p));
    if (p->kernel_variant != variant) ++p->generation;
    p->kernel_variant = variant;
    return XSDE_OK;
}

int xsde_kernel_variants(const xsde_problem *p) { return p ? variants_for(p) : 0; }

int xsde_set_scheme(xsde_problem *p, int32_t scheme) {
    if (!p) return fail(XSDE_EINVAL, "xsde_set_scheme: problem is NULL");
    if (scheme != XSDE_SCHEME_RK4IP && scheme != XSDE_SCHEME_SEMI_IMPLICIT)
        return fail(XSDE_EINVAL, "xsde_set_scheme: unknown scheme %d", scheme);
    if (p->scheme != scheme) {
        ++p->generation;
        p->table_dt = -1.0;   // the semi-implicit 2D step also needs whole-step tables
    }
    p->scheme = scheme;
    return XSDE_OK;
}

int xsde_set_nonlocal(xsde_problem *p, const double *khat) {
    if (!p) return fail(XSDE_EINVAL, "xsde_set_nonlocal: problem is NULL");
    if (!khat) {
        if (p->nonlocal) ++p->generation;
        p->nonlocal = false;
        return XSDE_OK;
    }
    if (p->grid.ndim < 1 || any_basis(p->grid))
        return fail(XSDE_EUNSUPPORTED,
                    "xsde_set_nonlocal: 1D, 2D and 3D Fourier lattices only (a circular convolution)");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device)
        return fail(XSDE_EINVAL, "xsde_set_nonlocal: current device %d is not the problem's %d", dev, p->device);
    const int64_t n = p->grid.npts;
    for (int64_t i = 0; i < 2 * n; ++i)
        if (!std::isfinite(khat[i])) return fail(XSDE_EINVAL, "xsde_set_nonlocal: non-finite kernel entry");
    const bool f32 = p->dtype == XSDE_C64;
    const size_t bytes = (size_t)n * (f32 ? sizeof(float2) : sizeof(double2));
    // the transforms of the kernels are unnormalised: fold the inverse's 1/N in
    std::vector<double> d(2 * n);
    std::vector<float> f(f32 ? 2 * n : 0);
    for (int64_t i = 0; i < 2 * n; ++i) {
        d[i] = khat[i] / (double)n;
        if (f32) f[i] = (float)d[i];
    }
    cudaError_t e = cudaDeviceSynchronize();   // no integration may still read the old kernel
    if (e == cudaSuccess && !p->d_knl) e = cudaMalloc(&p->d_knl, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_knl, f32 ? (const void *)f.data() : (const void *)d.data(), bytes,
                                         cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "xsde_set_nonlocal");
    p->nonlocal = true;
    ++p->generation;
    return XSDE_OK;
}

int xsde_probe_wait_timeout(xsde_problem *p, uint64_t wait_ns, void *stream) {
    if (!p) return fail(XSDE_EINVAL, "xsde_probe_wait_timeout: problem is NULL");
    if (wait_ns < 1000 || wait_ns > 1000000000ull)
        return fail(XSDE_EINVAL, "xsde_probe_wait_timeout: wait_ns %llu not in [1e3, 1e9]", (unsigned long long)wait_ns);
    XSDE_CUDA(launch_wait_timeout(wait_ns, p->d_status, static_cast<cudaStream_t>(stream)), "xsde_probe_wait_timeout");
    return XSDE_OK;
}

int xsde_measure_fma_peaks(double *fp32_tflops, double *fp64_tflops) {
    if (!fp32_tflops && !fp64_tflops) return fail(XSDE_EINVAL, "xsde_measure_fma_peaks: no output");
    if (measure_fma_peaks(fp32_tflops, fp64_tflops) != 0)
        return fail(XSDE_ECUDA, "xsde_measure_fma_peaks: %s", cudaGetErrorString(cudaGetLastError()));
    return XSDE_OK;
}

int xsde_set_noise_substeps(xsde_problem *p, int32_t substeps) {
    if (!p) return fail(XSDE_EINVAL, "xsde_set_noise_substeps: problem is NULL");
    if (substeps < 1 || substeps > 65536) return fail(XSDE_EINVAL, "xsde_set_noise_substeps: %d", substeps);
    if (p->noise_substeps != substeps) ++p->generation;
    p->noise_substeps = substeps;
    return XSDE_OK;
}


int xsde_profile(xsde_problem *p, int enable) {
    if (!p) return fail(XSDE_EINVAL, "xsde_profile: problem is NULL");
    if (!p->marks.empty()) {
        XSDE_CUDA(cudaDeviceSynchronize(), "xsde_profile");
        collect_marks(p);
    }
    p->profiling = enable != 0;
    for (int k = 0; k < XSDE_KERNEL_KINDS; ++k) {
        p->prof_ms[k] = 0.0;
        p->prof_launches[k] = 0;
    }
    return XSDE_OK;
}

int xsde_profile_report(xsde_problem *p, double *total_ms, int64_t *launches) {
    if (!p || !total_ms || !launches) return fail(XSDE_EINVAL, "xsde_profile_report: NULL argument");
    if (!p->marks.empty()) {
        for (auto &m : p->marks) XSDE_CUDA(cudaEventSynchronize(m.stop), "xsde_profile_report");
        collect_marks(p);
    }
    for (int k = 0; k < XSDE_KERNEL_KINDS; ++k) {
        total_ms[k] = p->prof_ms[k];
        launches[k] = p->prof_launches[k];
    }
    return XSDE_OK;
}

const char *xsde_kernel_name(int kind) {
    return (kind >= 0 && kind < XSDE_KERNEL_KINDS) ? kKernelNames[kind] : "";
}

int xsde_noise_philox(const uint32_t *counters, uint64_t seed, int64_t n, uint32_t *out, void *stream) {
    if (n < 0) return fail(XSDE_EINVAL, "xsde_noise_philox: n < 0");
    if (n > 0 && (!counters || !out)) return fail(XSDE_EINVAL, "xsde_noise_philox: NULL buffer");
    if (((uintptr_t)counters | (uintptr_t)out) % 16)
        return fail(XSDE_EINVAL, "xsde_noise_philox: buffers must be 16-byte aligned");
    XSDE_CUDA(launch_philox(counters, seed, n, out, static_cast<cudaStream_t>(stream)), "xsde_noise_philox");
    return XSDE_OK;
}

int xsde_noise_normals(const xsde_noise *noise, xsde_dtype dtype, int64_t npts, int64_t npaths,
                       int64_t path_offset, uint64_t step, void *out, void *stream) {
    if (!noise || !out) return fail(XSDE_EINVAL, "xsde_noise_normals: NULL argument");
    if (dtype != XSDE_C64 && dtype != XSDE_C128) return fail(XSDE_EINVAL, "xsde_noise_normals: unknown dtype");
    if (npts < 1 || npaths < 1 || path_offset < 0 || path_offset + npaths > (int64_t)UINT32_MAX + 1 ||
        npts > (int64_t)UINT32_MAX + 1 || step + 1 > (uint64_t)UINT32_MAX)
        return fail(XSDE_EINVAL, "xsde_noise_normals: indices out of the 32-bit counter range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = dtype == XSDE_C64
                        ? launch_normals<float>(noise->seed, npts, npaths, path_offset, (uint32_t)step, out, s)
                        : launch_normals<double>(noise->seed, npts, npaths, path_offset, (uint32_t)step, out, s);
    XSDE_CUDA(e, "xsde_noise_normals");
    return XSDE_OK;
}

int xsde_adjoint(xsde_problem *p, const xsde_vector *psi0, const xsde_vector *target, double dt, int64_t nsteps,
                 int32_t ckpt_every, double *loss, double *dLdV, void *dLdpsi0, void *stream) {
    if (!p || !psi0 || !target || !loss || !dLdV) return fail(XSDE_EINVAL, "xsde_adjoint: NULL argument");
    if (!p->have_ops) return fail(XSDE_EINVAL, "xsde_adjoint: operators not set");
    const xsde_grid &g = p->grid;
    if (g.ndim != 1 || g.n[0] < 256) return fail(XSDE_EUNSUPPORTED, "xsde_adjoint: 1D lattices of 256..2048 points");
    if (psi0->dtype != p->dtype || target->dtype != p->dtype)
        return fail(XSDE_EINVAL, "xsde_adjoint: field dtypes differ from the problem's");
    if (!same_lattice(psi0->grid, g) || !same_lattice(target->grid, g))
        return fail(XSDE_EINVAL, "xsde_adjoint: lattice differs");
    if (target->npaths != 1) return fail(XSDE_EINVAL, "xsde_adjoint: the target is a single field");
    if (p->noise.kind != XSDE_NOISE_NONE) return fail(XSDE_EUNSUPPORTED, "xsde_adjoint: deterministic problems only");
    if (p->scheme != XSDE_SCHEME_RK4IP) return fail(XSDE_EUNSUPPORTED, "xsde_adjoint: the adjoint of RK4IP only");
    if (p->nonlocal) return fail(XSDE_EUNSUPPORTED, "xsde_adjoint: the non-local term has no adjoint here");
    if (any_basis(g)) return fail(XSDE_EUNSUPPORTED, "xsde_adjoint: Fourier lattices only");
    if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 1 || ckpt_every < 1)
        return fail(XSDE_EINVAL, "xsde_adjoint: need dt > 0, nsteps >= 1, ckpt_every >= 1");
    if (p->N.pot_kind == XSDE_POT_TABLE && p->N.V_nt > 1 && nsteps > p->N.V_nt)
        return fail(XSDE_EINVAL, "xsde_adjoint: potential table has fewer rows than steps");
    const int64_t npaths = psi0->npaths;
    const int64_t K = ckpt_every < nsteps ? ckpt_every : nsteps;
    const int64_t nck = (nsteps + K - 1) / K;
    const size_t eb = elem_bytes(p->dtype);
    // all stage inputs kept (segments recomputed in parallel) when that takes at
    // most kAdjFullBytes; else one segment's at a time
    size_t full_limit = (size_t)2 << 30;
    if (const char *env = std::getenv("XSDE_ADJOINT_MAX_BYTES")) full_limit = (size_t)std::strtoull(env, nullptr, 10);
    const size_t full_need = (size_t)(nck + 4 * nsteps + 1) * npaths * g.npts * eb;
    const bool full = full_need <= full_limit && nck - 1 <= 65535;
    const size_t need = full ? full_need : (size_t)(nck + 4 * K) * npaths * g.npts * eb;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (p->adj_bytes < need) {
        if (p->d_adj) {
            XSDE_CUDA(cudaStreamSynchronize(s), "xsde_adjoint: workspace");
            cudaFree(p->d_adj);
            p->d_adj = nullptr;
            p->adj_bytes = 0;
        }
        XSDE_CUDA(cudaMalloc(&p->d_adj, need), "xsde_adjoint: workspace");
        p->adj_bytes = need;
    }
    XSDE_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s), "xsde_adjoint: memset");
    XSDE_CUDA(cudaMemsetAsync(dLdV, 0, (size_t)nsteps * g.npts * sizeof(double), s), "xsde_adjoint: memset");
    auto run = [&](auto tag) -> int {
        using R = decltype(tag);
        using V = cx<R>;
        int rc = ensure_tables<V>(p, dt, s);
        if (rc != XSDE_OK) return rc;
        AdjParams<R> q;
        Sampling sm;
        fill_terms<R>(p, dt, npaths, 0, q.lt, sm);
        q.psi0 = static_cast<const V *>(psi0->data);
        q.target = static_cast<const V *>(target->data);
        q.npaths = npaths;
        q.nsteps = nsteps;
        q.K = K;
        q.Etab = static_cast<const V *>(p->d_E[0]);
        // the problem's points-per-thread shape (the 2-point shape runs as 4);
        // at the default variant, fewer paths than SMs (one CTA per path, each
        // step a chain of dependent transforms) spread a path over 4 points per
        // thread, twice the threads of the 8-point shape
        int elems = rk4ip_1d_elems(p->kernel_variant) == 8 ? 8 : 4;
        if (p->kernel_variant == 0 && npaths < p->num_sms) elems = 4;
        q.tw = static_cast<const tw_t<R> *>(elems == 8 ? p->d_tw[0] : p->d_tw1d[0]);
        q.dx = grid_dx(g, 0);
        q.ckpt = static_cast<V *>(p->d_adj);
        q.interm = q.ckpt + (size_t)nck * npaths * g.npts;
        q.final_state = q.interm + (size_t)(full ? nsteps : K) * 4 * npaths * g.npts;
        q.loss = loss;
        q.dLdV = dLdV;
        q.dLdpsi0 = static_cast<V *>(dLdpsi0);
        q.status = p->d_status;
        q.interm_steps = full ? nsteps : K;
        const int phases[3] = {ADJ_FORWARD, ADJ_RECOMPUTE, ADJ_REVERSE};
        for (int i = 0; i < (full ? 3 : 1); ++i) {
            q.phase = full ? phases[i] : ADJ_SEQUENTIAL;
            XSDE_CUDA(timed(p, 1, s, [&] { return launch_adjoint_1d<R>(g.n[0], elems, q, s); }), "xsde_adjoint launch");
        }
        return XSDE_OK;
    };
    return p->dtype == XSDE_C64 ? run(0.0f) : run(0.0);
}

int xsde_integrate_adaptive(xsde_problem *p, xsde_vector *psi, const xsde_adaptive *spec, int64_t *accepted,
                            int64_t *rejected, void *stream) {
    if (!p || !psi || !spec || !accepted || !rejected)
        return fail(XSDE_EINVAL, "xsde_integrate_adaptive: NULL argument");
    if (!p->have_ops) return fail(XSDE_EINVAL, "xsde_integrate_adaptive: operators not set");
    if (psi->dtype != p->dtype) return fail(XSDE_EINVAL, "xsde_integrate_adaptive: field dtype differs");
    if (!same_lattice(psi->grid, p->grid)) return fail(XSDE_EINVAL, "xsde_integrate_adaptive: field lattice differs");
    const xsde_grid &g = p->grid;
    if (g.ndim != 1 || g.n[0] < 64)
        return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: 1D lattices of 64..2048 points");
    if (p->noise.kind != XSDE_NOISE_NONE)
        return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: deterministic problems only");
    if (p->N.pot_kind == XSDE_POT_TABLE && p->N.V_nt != 1)
        return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: a time-dependent potential table");
    if (p->samp.every > 0) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: sampling groups");
    if (p->nonlocal) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: the non-local term");
    if (any_basis(p->grid)) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: Fourier lattices only");
    if (!(spec->t_end >= 0.0) || !std::isfinite(spec->t_end) || !(spec->h0 > 0.0) || !std::isfinite(spec->h0) ||
        !std::isfinite(spec->tol) || spec->max_steps < 1 || (spec->picture != 0 && spec->picture != 1))
        return fail(XSDE_EINVAL, "xsde_integrate_adaptive: need t_end >= 0, h0 > 0, finite tol, max_steps >= 1");
    const int64_t npaths = psi->npaths;
    if (npaths > (int64_t)INT32_MAX) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_adaptive: too many paths");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != p->device) return fail(XSDE_EINVAL, "xsde_integrate_adaptive: wrong current device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = g.n[0];
    auto run = [&](auto zero) -> int {
        using R = decltype(zero);
        using V = cx<R>;
        int rc = p->table_dt > 0.0 ? XSDE_OK : ensure_tables<V>(p, 1.0, s);   // the twiddle tables
        if (rc != XSDE_OK) return rc;
        if ((rc = ensure_scratch(p, (size_t)6 * npaths * n * sizeof(V), s)) != XSDE_OK) return rc;
        AdaptiveParams<R> q;
        Sampling sm;
        fill_terms<R>(p, 1.0, npaths, 0, q.lt, sm);
        q.psi = static_cast<V *>(psi->data);
        q.npaths = npaths;
        const int elems = ark45_1d_elems(n);
        q.tw = static_cast<const tw_t<R> *>(elems == 8 ? p->d_tw[0] : p->d_tw1d[elems == 4 ? 0 : 1]);
        q.kbuf = static_cast<V *>(p->d_scratch);
        q.c0_re = p->L.c0_re;
        q.c0_im = p->L.c0_im;
        q.c2_re = p->L.c2_re;
        q.c2_im = p->L.c2_im;
        q.kscale = 2.0 * M_PI / (g.xmax[0] - g.xmin[0]);
        q.gnl = p->N.g;
        q.t_end = spec->t_end;
        q.tol = spec->tol;
        q.h0 = spec->h0;
        q.picture = spec->picture;
        q.max_steps = spec->max_steps;
        q.accepted = accepted;
        q.rejected = rejected;
        q.status = p->d_status;
        XSDE_CUDA(launch_ark45_1d<R>(n, q, s), "xsde_integrate_adaptive launch");
        return XSDE_OK;
    };
    return p->dtype == XSDE_C64 ? run(0.0f) : run(0.0);
}

int xsde_integrate_plain(xsde_problem *p, xsde_vector *psi, double dt, int64_t nsteps, int64_t npaths,
                         int64_t path_offset, uint64_t step_offset, void *stream) {
    int rc = check_integrate("xsde_integrate_plain", p, psi, dt, nsteps, npaths, path_offset, step_offset);
    if (rc != XSDE_OK) return rc;
    const xsde_grid &g = p->grid;
    if (g.ndim == 0) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_plain: 0D problems have no transform");
    if (p->samp.every > 0) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_plain: sampling groups are not supported");
    if (p->scheme != XSDE_SCHEME_RK4IP) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_plain: RK4IP only");
    if (p->nonlocal) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_plain: the non-local term");
    if (any_basis(p->grid)) return fail(XSDE_EUNSUPPORTED, "xsde_integrate_plain: Fourier lattices only");
    if (npaths * g.npts > (int64_t)INT32_MAX)
        return fail(XSDE_EUNSUPPORTED, "xsde_integrate_plain: more than 2^31 points per call");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp64 = p->dtype == XSDE_C128;
    const size_t eb = elem_bytes(p->dtype);
    const size_t field = (size_t)npaths * g.npts * eb;
    if (!plain_plan_matches(p->plain, g.ndim, g.n, npaths, fp64)) {
        XSDE_CUDA(cudaStreamSynchronize(s), "xsde_integrate_plain");
        plain_plan_destroy(p->plain);
        p->plain = nullptr;
        XSDE_CUDA(plain_plan_create(g.ndim, g.n, npaths, fp64, &p->plain), "xsde_integrate_plain: cuFFT plan");
    }
    if (p->plain_bytes < 4 * field) {
        XSDE_CUDA(cudaStreamSynchronize(s), "xsde_integrate_plain");
        cudaFree(p->d_plain);
        p->d_plain = nullptr;
        p->plain_bytes = 0;
        XSDE_CUDA(cudaMalloc(&p->d_plain, 4 * field), "xsde_integrate_plain: work fields");
        p->plain_bytes = 4 * field;
    }
    if (p->plain_dt != dt || p->plain_gen != p->generation || !p->d_plain_E) {
        // exp((c0 + c2 |k|^2) dt/2) / npts in FP64, rounded once
        const std::complex<double> c0(p->L.c0_re, p->L.c0_im), c2(p->L.c2_re, p->L.c2_im);
        std::vector<std::complex<double>> e((size_t)g.npts);
        for (int64_t j = 0; j < g.npts; ++j) {
            int64_t r = j;
            double k2 = 0.0;
            for (int d = g.ndim - 1; d >= 0; --d) {
                const double k = kval(g, d, (int)(r % g.n[d]));
                k2 += k * k;
                r /= g.n[d];
            }
            e[(size_t)j] = std::exp((c0 + c2 * k2) * (0.5 * dt)) / (double)g.npts;
        }
        XSDE_CUDA(cudaStreamSynchronize(s), "xsde_integrate_plain");
        cudaFree(p->d_plain_E);
        p->d_plain_E = nullptr;
        XSDE_CUDA(cudaMalloc(&p->d_plain_E, (size_t)g.npts * eb), "xsde_integrate_plain: table");
        if (fp64) {
            std::vector<double2> h((size_t)g.npts);
            for (size_t j = 0; j < h.size(); ++j) h[j] = make_double2(e[j].real(), e[j].imag());
            XSDE_CUDA(cudaMemcpy(p->d_plain_E, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice),
                      "xsde_integrate_plain: table");
        } else {
            std::vector<float2> h((size_t)g.npts);
            for (size_t j = 0; j < h.size(); ++j) h[j] = make_float2((float)e[j].real(), (float)e[j].imag());
            XSDE_CUDA(cudaMemcpy(p->d_plain_E, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice),
                      "xsde_integrate_plain: table");
        }
        p->plain_dt = dt;
        p->plain_gen = p->generation;
    }
    auto run = [&](auto zero) -> int {
        using R = decltype(zero);
        using V = cx<R>;
        PlainParams<R> q;
        LocalTerm<R> lt;
        Sampling sm;
        fill_terms<R>(p, dt, npaths, path_offset, lt, sm);
        V *w = static_cast<V *>(p->d_plain);
        const int64_t n = npaths * g.npts;
        q.a = static_cast<V *>(psi->data);
        q.aI = w;
        q.k = w + n;
        q.acc = w + 2 * n;
        q.tmp = w + 3 * n;
        q.E = static_cast<const V *>(p->d_plain_E);
        q.npaths = npaths;
        q.npts = g.npts;
        q.ndim = g.ndim;
        for (int d = 0; d < 3; ++d) q.n[d] = d < g.ndim ? g.n[d] : 1;
        q.nsteps = nsteps;
        q.step0 = step_offset;
        q.lt = lt;
        XSDE_CUDA(run_plain<R>(p->plain, q, p->num_sms, s), "xsde_integrate_plain");
        return XSDE_OK;
    };
    return fp64 ? run(0.0) : run(0.0f);
}

int xsde_synchronize(xsde_problem *p, void *stream) {
    if (!p) return fail(XSDE_EINVAL, "xsde_synchronize: problem is NULL");
    XSDE_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "xsde_synchronize");
    int st = 0;
    XSDE_CUDA(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost), "xsde_synchronize: status");
    if (st) XSDE_CUDA(cudaMemset(p->d_status, 0, sizeof(int)), "xsde_synchronize: reset");
    if (st & ST_TIMEOUT) return fail(XSDE_ETIMEOUT, "a bounded device-side wait gave up");
    if (st & ST_NONFINITE) return fail(XSDE_ENONFINITE, "the field became non-finite");
    if (st & ST_STEP_LIMIT) return fail(XSDE_ELIMIT, "an adaptive path used up its step attempts");
    if (st & ST_BOUNDS) return fail(XSDE_EBOUNDS, "an index left its buffer (bounds-checking build)");
    return XSDE_OK;
}

}  // extern "C"

// ===========================================================================
// Autotuning and batches of uneven instances (the paper's many paths and
// independent simulations, Secs. 2.5 and 3, gathered into one launch).
//
// A lattice offers a few kernel variants that compute the same scheme with
// different launch shapes: 1D, the number of paths one CTA carries; 2D
// complex64, the persistent TMA-pipelined passes or the generic tiles.
// xsde_autotune times each on a copy of the caller's field and keeps the
// fastest.  A batch binds several problems to their fields and records all
// their pass schedules as one CUDA graph: one host launch replays the whole
// batch; the single-kernel 0D / 1D members are concurrent branches, the 2D / 3D
// members (each thousands of passes over every SM) follow one another.
// ===========================================================================
struct xsde_batch {
    int device = -1;
    int flags = 0;
    bool tuned = false;
    std::vector<xsde_batch_member> m;
    cudaStream_t cap = nullptr;               // capture origin
    std::vector<cudaStream_t> streams;        // one branch per member
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec = nullptr;
    // what the instantiated graph was recorded for
    double dt = -1.0;
    int64_t nsteps = -1;
    uint64_t step0 = 0;
    std::vector<std::vector<uintptr_t>> sig;
};

namespace {

std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;
bool g_tune_file_loaded = false;

const char *tune_cache_path() {
    const char *path = std::getenv("XSDE_AUTOTUNE_CACHE");
    return (path && *path) ? path : nullptr;
}

std::string tune_key(const xsde_problem *p, int64_t npaths) {
    char name[256] = "unknown";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) snprintf(name, sizeof name, "%s", prop.name);
    for (char *c = name; *c; ++c)
        if (*c == ' ' || *c == '\t') *c = '_';
    char buf[512];
    snprintf(buf, sizeof buf, "%s/sm%d/%s/d%d/%dx%dx%d/p%lld", name, p->num_sms, p->dtype == XSDE_C64 ? "c64" : "c128",
             p->grid.ndim, p->grid.n[0], p->grid.ndim > 1 ? p->grid.n[1] : 1, p->grid.ndim > 2 ? p->grid.n[2] : 1,
             (long long)npaths);
    return buf;
}

// lines "key variant"; later lines win
void tune_file_load_locked() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char *path = tune_cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[512];
    int v = 0;
    while (std::fscanf(f, "%511s %d", key, &v) == 2) g_tune_cache[key] = v;
    std::fclose(f);
}

void tune_file_append_locked(const std::string &key, int v) {
    const char *path = tune_cache_path();
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d\n", key.c_str(), v);
    std::fclose(f);
}

int tune_problem(xsde_problem *p, const xsde_vector *psi, double dt, int64_t nsteps, bool reuse, int *best_out,
                 double *ms_out, cudaStream_t s) {
    const int nv = variants_for(p);
    const std::string key = tune_key(p, psi->npaths);
    if (reuse) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_file_load_locked();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end() && it->second >= 0 && it->second < nv) {
            if (p->kernel_variant != it->second) ++p->generation;
            p->kernel_variant = it->second;
            if (best_out) *best_out = it->second;
            return XSDE_OK;
        }
    }
    // a time-dependent potential table bounds the steps that can be taken
    if (p->N.pot_kind == XSDE_POT_TABLE && p->N.V_nt > 1) nsteps = std::min<int64_t>(nsteps, p->N.V_nt);
    const size_t bytes = (size_t)psi->npaths * psi->grid.npts * elem_bytes(p->dtype);
    void *tmp = nullptr;
    XSDE_CUDA(cudaMalloc(&tmp, bytes ? bytes : 16), "xsde_autotune: field copy");
    // sampling and profiling are suspended while tuning
    const xsde_sampling samp = p->samp;
    double *const per_path = p->per_path, *const per_point = p->per_point;
    const bool profiling = p->profiling;
    const int old_variant = p->kernel_variant;
    p->samp = xsde_sampling{0, 0};
    p->per_path = p->per_point = nullptr;
    p->profiling = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int rc = XSDE_OK;
    cudaError_t e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    if (e != cudaSuccess) rc = cuda_fail(e, "xsde_autotune: events");
    int best = 0;
    double best_ms = 0.0;
    for (int v = 0; v < nv && rc == XSDE_OK; ++v) {
        p->kernel_variant = v;
        double vmin = INFINITY;
        for (int rep = 0; rep < 4 && rc == XSDE_OK; ++rep) {   // rep 0 warms up
            e = cudaMemcpyAsync(tmp, psi->data, bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaEventRecord(ev0, s);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "xsde_autotune");
                break;
            }
            rc = integrate_on(p, tmp, dt, nsteps, psi->npaths, 0, 0, s);
            if (rc != XSDE_OK) break;
            e = cudaEventRecord(ev1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "xsde_autotune: timing");
                break;
            }
            if (rep > 0) vmin = std::min(vmin, (double)ms);
        }
        if (rc != XSDE_OK) break;
        if (ms_out) ms_out[v] = vmin;
        if (v == 0 || vmin < best_ms) {
            best_ms = vmin;
            best = v;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(tmp);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    p->samp = samp;
    p->per_path = per_path;
    p->per_point = per_point;
    p->profiling = profiling;
    if (rc != XSDE_OK) {
        p->kernel_variant = old_variant;
        return rc;
    }
    if (best != old_variant) ++p->generation;
    p->kernel_variant = best;
    if (best_out) *best_out = best;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_file_load_locked();
    auto it = g_tune_cache.find(key);
    if (it == g_tune_cache.end() || it->second != best) {
        g_tune_cache[key] = best;
        tune_file_append_locked(key, best);
    }
    return XSDE_OK;
}

// Tables for dt and the scratch field, made ready outside any capture.
int prepare_member(xsde_problem *p, double dt, int64_t npaths, cudaStream_t s) {
    int rc = p->dtype == XSDE_C64 ? ensure_tables<cx<float>>(p, dt, s) : ensure_tables<cx<double>>(p, dt, s);
    if (rc == XSDE_OK && p->grid.ndim >= 2)
        rc = ensure_scratch(p, (size_t)scratch_fields(p) * npaths * p->grid.npts * elem_bytes(p->dtype), s);
    return rc;
}

// Everything a recorded launch sequence depends on besides (dt, nsteps, step0).
std::vector<uintptr_t> member_signature(const xsde_batch_member &m) {
    const xsde_problem *p = m.prob;
    std::vector<uintptr_t> v = {(uintptr_t)p->generation, (uintptr_t)m.psi->data, (uintptr_t)p->d_scratch,
                                (uintptr_t)m.psi->npaths, (uintptr_t)m.path_offset};
    for (int d = 0; d < 3; ++d) {
        v.push_back((uintptr_t)p->d_tw[d]);
        v.push_back((uintptr_t)p->d_E[d]);
    }
    v.push_back((uintptr_t)p->d_tw1d[0]);
    v.push_back((uintptr_t)p->d_tw1d[1]);
    for (int d = 0; d < 3; ++d) v.push_back((uintptr_t)p->d_tw2[d]);
    v.push_back((uintptr_t)p->d_twp);
    return v;
}

void batch_release(xsde_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    for (cudaStream_t st : b->streams)
        if (st) cudaStreamDestroy(st);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

// Record every member's schedule as one branch of a graph and instantiate it
// (or update the existing executable graph in place).
int batch_capture(xsde_batch *b, double dt, int64_t nsteps, uint64_t step0) {
    const size_t n = b->m.size();
    std::vector<bool> profiling(n);
    for (size_t i = 0; i < n; ++i) {
        profiling[i] = b->m[i].prob->profiling;
        b->m[i].prob->profiling = false;   // no event pairs inside the graph
    }
    cudaGraph_t graph = nullptr;
    int rc = XSDE_OK;
    // 0D / 1D members are one whole-run kernel each: they run as concurrent
    // branches, so their CTAs share the waves of the GPU.  2D / 3D members are
    // thousands of persistent passes that size their grids to every SM and
    // hand out work statically; a pass that has to share SMs with long-running
    // CTAs of another member finishes with its slowest CTA, so these members
    // follow one another on the capture stream after the concurrent branches.
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = cudaEventRecord(b->fork, b->cap);
        for (size_t i = 0; i < n && e == cudaSuccess && rc == XSDE_OK; ++i) {
            const xsde_batch_member &m = b->m[i];
            if (m.prob->grid.ndim >= 2) continue;
            e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
            if (e != cudaSuccess) break;
            rc = integrate_on(m.prob, m.psi->data, dt, nsteps, m.psi->npaths, m.path_offset, step0, b->streams[i]);
            if (rc != XSDE_OK) break;
            e = cudaEventRecord(b->join[i], b->streams[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[i], 0);
        }
        for (size_t i = 0; i < n && e == cudaSuccess && rc == XSDE_OK; ++i) {
            const xsde_batch_member &m = b->m[i];
            if (m.prob->grid.ndim < 2) continue;
            rc = integrate_on(m.prob, m.psi->data, dt, nsteps, m.psi->npaths, m.path_offset, step0, b->cap);
        }
        const cudaError_t e_end = cudaStreamEndCapture(b->cap, &graph);
        if (e == cudaSuccess) e = e_end;
    }
    for (size_t i = 0; i < n; ++i) b->m[i].prob->profiling = profiling[i];
    if (rc != XSDE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != XSDE_OK ? rc : cuda_fail(e, "xsde_batch_integrate: graph capture");
    }
    if (b->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(b->exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(b->exec);
            b->exec = nullptr;
        }
    }
    if (!b->exec) e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return cuda_fail(e, "xsde_batch_integrate: graph instantiate");
    }
    b->dt = dt;
    b->nsteps = nsteps;
    b->step0 = step0;
    b->sig.resize(n);
    for (size_t i = 0; i < n; ++i) b->sig[i] = member_signature(b->m[i]);
    return XSDE_OK;
}

}  // namespace

extern "C" {

int xsde_autotune(xsde_problem *p, const xsde_vector *psi, double dt, int64_t nsteps, int *best, double *ms,
                  void *stream) {
    if (!psi) return fail(XSDE_EINVAL, "xsde_autotune: field is NULL");
    if (nsteps < 1) return fail(XSDE_EINVAL, "xsde_autotune: nsteps must be >= 1");
    const int rc = check_integrate("xsde_autotune", p, psi, dt, nsteps, psi->npaths, 0, 0);
    if (rc != XSDE_OK) return rc;
    return tune_problem(p, psi, dt, nsteps, ms == nullptr, best, ms, static_cast<cudaStream_t>(stream));
}

int xsde_batch_create(const xsde_batch_member *members, int n, int flags, xsde_batch **out) {
    if (!out) return fail(XSDE_EINVAL, "xsde_batch_create: out is NULL");
    *out = nullptr;
    if (!members || n < 1) return fail(XSDE_EINVAL, "xsde_batch_create: no members");
    if (flags & ~XSDE_BATCH_AUTOTUNE) return fail(XSDE_EINVAL, "xsde_batch_create: unknown flags 0x%x", flags);
    int dev = -1;
    cudaGetDevice(&dev);
    for (int i = 0; i < n; ++i) {
        const xsde_batch_member &m = members[i];
        if (!m.prob || !m.psi) return fail(XSDE_EINVAL, "xsde_batch_create: member %d has a NULL problem or field", i);
        if (m.prob->device != dev)
            return fail(XSDE_EINVAL, "xsde_batch_create: member %d lives on device %d, not the current %d", i,
                        m.prob->device, dev);
        for (int j = 0; j < i; ++j) {
            if (members[j].prob == m.prob)
                return fail(XSDE_EINVAL, "xsde_batch_create: members %d and %d share a problem (its scratch)", j, i);
            if (members[j].psi->data == m.psi->data)
                return fail(XSDE_EINVAL, "xsde_batch_create: members %d and %d share a field", j, i);
        }
    }
    xsde_batch *b = new (std::nothrow) xsde_batch();
    if (!b) return fail(XSDE_ENOMEM, "xsde_batch_create: out of host memory");
    b->device = dev;
    b->flags = flags;
    b->m.assign(members, members + n);
    b->streams.assign(n, nullptr);
    b->join.assign(n, nullptr);
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        batch_release(b);
        return cuda_fail(e, "xsde_batch_create");
    }
    *out = b;
    return XSDE_OK;
}

int xsde_batch_integrate(xsde_batch *b, double dt, int64_t nsteps, uint64_t step_offset, void *stream) {
    if (!b) return fail(XSDE_EINVAL, "xsde_batch_integrate: batch is NULL");
    int rc;
    for (const xsde_batch_member &m : b->m)
        if ((rc = check_integrate("xsde_batch_integrate", m.prob, m.psi, dt, nsteps, m.psi->npaths, m.path_offset,
                                  step_offset)) != XSDE_OK)
            return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((b->flags & XSDE_BATCH_AUTOTUNE) && !b->tuned) {
        const int64_t probe = std::max<int64_t>(1, std::min<int64_t>(nsteps, 10));
        for (const xsde_batch_member &m : b->m)
            if ((rc = tune_problem(m.prob, m.psi, dt, probe, true, nullptr, nullptr, s)) != XSDE_OK) return rc;
        b->tuned = true;
    }
    for (const xsde_batch_member &m : b->m)
        if ((rc = prepare_member(m.prob, dt, m.psi->npaths, s)) != XSDE_OK) return rc;
    bool stale = !b->exec || b->dt != dt || b->nsteps != nsteps || b->step0 != step_offset;
    for (size_t i = 0; i < b->m.size() && !stale; ++i) stale = b->sig[i] != member_signature(b->m[i]);
    if (stale) {
        // an update must not race a replay of the previous graph
        if (b->exec) XSDE_CUDA(cudaStreamSynchronize(s), "xsde_batch_integrate");
        if ((rc = batch_capture(b, dt, nsteps, step_offset)) != XSDE_OK) return rc;
    }
    XSDE_CUDA(cudaGraphLaunch(b->exec, s), "xsde_batch_integrate: graph launch");
    return XSDE_OK;
}

void xsde_batch_destroy(xsde_batch *b) {
    if (!b) return;
    cudaDeviceSynchronize();
    batch_release(b);
}

}  // extern "C"

// ===========================================================================
// Integration that allocates nothing (the paper has no counterpart).
//
// Some callers cannot allocate device memory at the point where they
// integrate: code that runs under a fixed memory budget or a caller-owned
// pool (every byte is accounted for up front), real-time loops in which a
// cudaMalloc/cudaFree would stall on a device-wide synchronisation, and hosts
// that hand this library a problem and device pointers but no permission to
// grow the device heap.  xsde_integrate_static_scratch serves them on 2D
// lattices: instead of the problem's own scratch field and Fourier tables it
// uses file-scope device arrays that every GPU loading the library holds
// until process exit (kStaticScratchBytes for the scratch field plus
// kStaticTableBytes for the tables).
// ===========================================================================
namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;     // 16 MiB scratch field
constexpr int kStaticMaxN = 2048;                             // longest dimension
constexpr size_t kStaticTwBytes = (size_t)kStaticMaxN * 16;   // twiddles of one dimension
constexpr size_t kStaticEBytes = (size_t)2 * kStaticMaxN * 16; // exp(L dt/2) hi+lo of one dimension
constexpr size_t kStaticTableBytes = 2 * (kStaticTwBytes + kStaticEBytes);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
static __device__ __align__(256) unsigned char g_static_tables[kStaticTableBytes];

// Device addresses of the two arrays, resolved once per device.  In host code
// the array names are host-side stand-ins, never device addresses.
struct StaticArrays {
    void *scratch = nullptr;
    unsigned char *tables = nullptr;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
StaticArrays g_static_arrays[kMaxDevices];
std::mutex g_static_mutex;

int static_arrays_for(int dev, StaticArrays **out) {
    if (dev < 0 || dev >= kMaxDevices)
        return fail(XSDE_EUNSUPPORTED, "xsde_integrate_static_scratch: device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_static_mutex);
    StaticArrays &sa = g_static_arrays[dev];
    if (!sa.ready) {
        void *scratch = nullptr, *tables = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&scratch, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "xsde_integrate_static_scratch: scratch address");
        e = cudaGetSymbolAddress(&tables, g_static_tables);
        if (e != cudaSuccess) return cuda_fail(e, "xsde_integrate_static_scratch: table address");
        sa.scratch = scratch;
        sa.tables = static_cast<unsigned char *>(tables);
        sa.ready = true;
    }
    *out = &sa;
    return XSDE_OK;
}

// host staging of the tables (per thread, no heap)
thread_local unsigned char t_host_tables[kStaticTableBytes];

template <typename R>
int static_integrate(xsde_problem *p, void *psi, double dt, int64_t nsteps, int64_t npaths, int64_t path_offset,
                     uint64_t step0, cudaStream_t s, const StaticArrays &sa) {
    using V = cx<R>;
    const xsde_grid &g = p->grid;
    const std::complex<double> c0(p->L.c0_re, p->L.c0_im), c2(p->L.c2_re, p->L.c2_im);
    // tables into the host staging area, same layouts as the problem's own tables
    unsigned char *hdim[2] = {t_host_tables, t_host_tables + kStaticTwBytes + kStaticEBytes};
    for (int d = 0; d < 2; ++d) {
        const int n = g.n[d];
        tw_t<R> *tw = reinterpret_cast<tw_t<R> *>(hdim[d]);
        V *e = reinterpret_cast<V *>(hdim[d] + kStaticTwBytes);
        make_twiddle(std::complex<double>(0.0, 0.0), &tw[n - 1]);
        for (int ns = 1; ns < n;) {
            const int rad = stage_radix<8>(n / ns);
            if (ns > 1) {
                const int off = stage_table_offset(n, ns);
                for (int r = 1; r < rad; ++r)
                    for (int k = 0; k < ns; ++k) {
                        const long m = (long)r * k * (n / (ns * rad));
                        make_twiddle(std::polar(1.0, -2.0 * M_PI * (double)m / n), &tw[off + (r - 1) * ns + k]);
                    }
            }
            ns *= rad;
        }
        for (int i = 0; i < n; ++i) {
            const double k = kval(g, d, i);
            const std::complex<double> v =
                d == 0 ? std::exp((c0 + c2 * (k * k)) * (0.5 * dt)) / ((double)g.n[0] * g.n[1])
                       : std::exp(c2 * (k * k) * (0.5 * dt));
            split_hi_lo(v, &e[i], &e[n + i]);
        }
    }
    XSDE_CUDA(cudaMemcpyAsync(sa.tables, t_host_tables, kStaticTableBytes, cudaMemcpyHostToDevice, s),
              "xsde_integrate_static_scratch: tables");
    XSDE_CUDA(cudaStreamSynchronize(s), "xsde_integrate_static_scratch: tables");

    LocalTerm<R> lt;
    Sampling sm;
    fill_terms<R>(p, dt, npaths, path_offset, lt, sm);
    const bool sampling = sm.every > 0;
    sm.nsamp = sampling ? nsteps / sm.every + 1 : 0;
    if (sampling) {
        const int64_t nsamp = nsteps / sm.every + 1;
        if (sm.per_path && (sm.which & (MOM_NORM | MOM_ENERGY)))
            XSDE_CUDA(cudaMemsetAsync(sm.per_path, 0, (size_t)nsamp * npaths * 2 * sizeof(double), s), "memset");
        if (sm.per_point && (sm.which & (MOM_MOD2 | MOM_MOD4)))
            XSDE_CUDA(cudaMemsetAsync(sm.per_point, 0, (size_t)nsamp * g.npts * 2 * sizeof(double), s), "memset");
    }
    Params2D<R> q;
    q.A = static_cast<V *>(psi);
    q.B = static_cast<V *>(sa.scratch);   // fully written by the first pass before it is read
    q.npaths = npaths;
    q.n0 = g.n[0];
    q.n1 = g.n[1];
    q.tw0 = reinterpret_cast<const tw_t<R> *>(sa.tables);
    q.E0 = reinterpret_cast<const V *>(sa.tables + kStaticTwBytes);
    q.tw1 = reinterpret_cast<const tw_t<R> *>(sa.tables + kStaticTwBytes + kStaticEBytes);
    q.E1 = reinterpret_cast<const V *>(sa.tables + 2 * kStaticTwBytes + kStaticEBytes);
    q.lt = lt;
    q.sm = sm;
    q.status = p->d_status;
    const int S = sm.every;
    auto row = [&](int mode, uint64_t sg, int slot) {
        q.sg = sg;
        q.sample_slot = slot;
        return launch_row_pass<R>(mode, q, s);
    };
    auto col = [&](int mode, int slot) {
        q.sample_slot = slot;
        return launch_col_pass<R>(mode, q, s);
    };
    if (nsteps > 0) {
        XSDE_CUDA(row(ROW_PROLOGUE, step0, sampling ? 0 : -1), "row pass");
        for (int64_t n = 0; n < nsteps; ++n) {
            const uint64_t sg = step0 + n;
            XSDE_CUDA(col(COL_PROPAGATE, (sampling && n % S == 0) ? (int)(n / S) : -1), "col pass");
            XSDE_CUDA(row(ROW_STAGE2, sg, -1), "row pass");
            XSDE_CUDA(col(COL_PROPAGATE, -1), "col pass");
            if (n + 1 < nsteps) {
                const int slot = (sampling && (n + 1) % S == 0) ? (int)((n + 1) / S) : -1;
                XSDE_CUDA(row(ROW_STEADY, sg, slot), "row pass");
            } else {
                XSDE_CUDA(row(ROW_EPILOGUE, sg, -1), "row pass");
            }
        }
    }
    if (sampling && nsteps % S == 0) {
        const int slot = (int)(nsteps / S);
        XSDE_CUDA(row(ROW_FFT_ONLY, step0 + nsteps, slot), "row pass");
        XSDE_CUDA(col(COL_SPECTRAL, slot), "col pass");
    }
    return XSDE_OK;
}

}  // namespace

extern "C" int xsde_integrate_static_scratch(xsde_problem *p, xsde_vector *psi, double dt, int64_t nsteps,
                                             int64_t npaths, int64_t path_offset, uint64_t step_offset,
                                             void *stream) {
    const char *who = "xsde_integrate_static_scratch";
    // the argument checks of xsde_integrate (field, dt, 32-bit path and step
    // counters including noise substeps, potential table rows, current device)
    int rc = check_integrate(who, p, psi, dt, nsteps, npaths, path_offset, step_offset);
    if (rc != XSDE_OK) return rc;
    if (p->grid.ndim != 2) return fail(XSDE_EUNSUPPORTED, "%s: only 2D lattices use a scratch field", who);
    if (any_basis(p->grid)) return fail(XSDE_EUNSUPPORTED, "%s: Fourier lattices only", who);
    // the static path runs the RK4IP pass schedule with local terms only
    if (p->scheme != XSDE_SCHEME_RK4IP)
        return fail(XSDE_EUNSUPPORTED, "%s: the RK4IP scheme only (the semi-implicit scheme: xsde_integrate)", who);
    if (p->nonlocal) return fail(XSDE_EUNSUPPORTED, "%s: no non-local term (use xsde_integrate)", who);
    const size_t need = (size_t)npaths * p->grid.npts * elem_bytes(p->dtype);
    if (need > kStaticScratchBytes)
        return fail(XSDE_EINVAL,
                    "%s: the scratch field needs %zu bytes, more than the %zu-byte static buffer (npaths x points "
                    "x element size); use xsde_integrate or fewer paths per call",
                    who, need, kStaticScratchBytes);
    const int dev = p->device;
    StaticArrays *sa = nullptr;
    rc = static_arrays_for(dev, &sa);
    if (rc != XSDE_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return p->dtype == XSDE_C64
               ? static_integrate<float>(p, psi->data, dt, nsteps, npaths, path_offset, step_offset, s, *sa)
               : static_integrate<double>(p, psi->data, dt, nsteps, npaths, path_offset, step_offset, s, *sa);
}
