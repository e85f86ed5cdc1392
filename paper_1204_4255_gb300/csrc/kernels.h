// kernels.h -- parameter blocks and launchers of the RK4IP kernels (internal).
//
// Equation family (XMDS2 Sec. 2.6, Eq. PDEBeforeIPTransform):
//   d psi/dt = L psi + g,  L(k) = c0 + c2|k|^2  (applied as exp(L dt/2) in Fourier space)
//   N(u) = dt g = dt * [-i (V(x,t) + g_nl |u|^2 + alpha xi_r) u + sigma xi_a]  (real space)
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "bounds.cuh"
#include "device_common.cuh"
#include "fft.cuh"

namespace xsde {

enum PotMode { PM_NONE = 0, PM_HARMONIC = 1, PM_TABLE = 2 };
enum NoiseMode { NM_NONE = 0, NM_ADD_REAL = 1, NM_ADD_COMPLEX = 2, NM_MUL_REAL = 3 };

// status bits written by kernels into the problem's device error word
enum { ST_NONFINITE = 1, ST_TIMEOUT = 2 };

// The real-space term: potential, nonlinearity and noise of one step.
template <typename R> struct LocalTerm {
    R dt;                 // time step
    R gdt;                // g_nl * dt
    int pot;              // PotMode
    R hw2[3];             // omega_d^2 / 2
    R xmin[3], dx[3];     // lattice origin and spacing (working precision)
    const R *V;           // [V_nt][npts] raw potential (PM_TABLE)
    int64_t V_nt;
    int64_t npts;
    int noise;            // NoiseMode
    R nscale;             // amplitude * sqrt(dt/dV)   (complex noise: / sqrt 2)
    uint2 key;            // Philox key (seed_lo, seed_hi)
    int64_t path_offset;  // global index of local path 0
    int substeps = 1;     // a step's noise is the mean of this many finer steps' (see point_term)
    int *status = nullptr;  // device error word (index checks of the bounds-checking build)
};

// Sampling group: FP64 per-path (norm, energy) and per-point (mean |psi|^2, |psi|^4).
struct Sampling {
    int every;             // 0: off
    int which;             // XSDE_MOM_* bits
    double *per_path;      // [nsamp][npaths][2]
    double *per_point;     // [nsamp][npts][2]
    double dV;
    double inv_paths;      // 1/npaths (means over paths)
    double h0, h2;         // Re(i L(k)) = h0 + h2 |k|^2 (kinetic energy density)
    double kscale[3];      // 2 pi / (xmax - xmin) per dimension
    double g;              // g_nl (interaction energy g/2 |psi|^4)
    int64_t nsamp = 0;     // samples of the call (extent of per_path / per_point)
};

enum { MOM_NORM = 1, MOM_ENERGY = 2, MOM_MOD2 = 4, MOM_MOD4 = 8 };

// --------------------------------------------------------------------------
// 1D: one CTA slot per path runs every step with the field in registers.
// --------------------------------------------------------------------------
template <typename R> struct Params1D {
    cx<R> *psi;            // [npaths][N] real space, in/out
    int64_t npaths;
    int64_t nsteps;
    uint64_t step0;        // global index of local step 0
    const cx<R> *Etab;     // exp(L(k) dt/2)/N in FFT order, hi [N] then lo [N]
    const tw_t<R> *tw;     // per-stage twiddles of the variant's radix plan [N] (FP32: hi, lo)
    LocalTerm<R> lt;
    Sampling sm;
    int *status;
    int scheme = 0;        // 0 RK4IP, 1 semi-implicit midpoint (default launch shape only)
    const cx<R> *knl = nullptr;   // non-local kernel khat/N in FFT order [N], or none
                                  // (RK4IP at the default launch shape only)
    int basis = 0;         // 0 Fourier; 1 / 2 cosine / sine lattice (default launch shape
                           // only): Etab holds A and Btab B of U_k = A_k V_k + B_k V_{N-k}
    const cx<R> *Btab = nullptr;   // hi [N] then lo [N]
};
// variant v in [0, rk4ip_1d_variants()) sets the launch shape: elements per
// thread rk4ip_1d_elems(v) (8, or 4 / 2 for variants 4 / 5, whose twiddle
// table follows the radix-4 / radix-2 plan) and paths per CTA (variants 0-3:
// the default filling 128 threads, a half, a quarter, twice)
// FP32 / FP64 FMA throughput of the current device (TFLOP/s); 0 or -1
int measure_fma_peaks(double *fp32_tflops, double *fp64_tflops);
// one CTA whose bounded wait on a barrier nobody arrives at runs out (ST_TIMEOUT)
cudaError_t launch_wait_timeout(uint64_t wait_ns, int *status, cudaStream_t s);
int rk4ip_1d_variants();
int rk4ip_1d_elems(int variant);
template <typename R> cudaError_t launch_rk4ip_1d(int n, int variant, const Params1D<R> &p, cudaStream_t s);

// --------------------------------------------------------------------------
// 2D: row passes (contiguous dimension 1, real-space work) and column passes
// (dimension 0, exp(L dt/2)); fields between passes are FFT'd along dim 1.
// --------------------------------------------------------------------------
enum RowMode {
    ROW_PROLOGUE = 0,   // psi (real) -> A = F1 psi, B = F1 N(psi)
    ROW_STAGE2 = 1,     // A = a_I, B = k1 -> A = u1 = a_I + k3, B = a_I + k1/6 + k2/3 + k3/3
    ROW_STEADY = 2,     // A = D u1, B = D acc -> a' = D acc + N(D u1)/6; A = F1 a', B = F1 N(a')
    ROW_EPILOGUE = 3,   // as STEADY but writes a' in real space to A only
    ROW_FFT_ONLY = 4,   // A (real) -> B = F1 A (for the spectral part of the energy)
    ROW_SI = 5,         // semi-implicit scheme on A alone; sub-operation p.si_op (SiOp)
    ROW_NL = 6          // RK4IP with a non-local pair potential; sub-operation p.nl_op (NlOp)
};
// RK4IP steps with a non-local potential V_nl[u] = Re F^-1[khat F |u|^2] on 2D
// lattices evaluate every N(u) with the V_nl of its own argument, so each
// evaluation waits for a density convolution: a row pass forms C = F1 |u|^2, a
// column pass (COL_CONV) takes C to F1 V_nl, and the next row pass reads V_nl
// as Re F1^-1 C.  Fields between passes (A, B as in RowMode; D real space):
enum NlOp {
    NL_DENSITY = 0,     // A (real u) -> C = F1 |u|^2
    NL_PROLOGUE = 1,    // A (real a), C -> A = E1 F1 a, B = E1 F1 N(a) (at step sg; sample of a)
    NL_FFT = 2,         // A (real a), C -> sample of a (local terms with V_nl), B = F1 a
    NL_S2A = 3,         // A = F1 a_I, B = F1 k1 -> C = F1 |a_I + k1/2|^2
    NL_S2B = 4,         // A, B, C -> D = k2 = N(a_I + k1/2), C = F1 |a_I + k2/2|^2
    NL_S2C = 5,         // A, B, C, D -> k3; A = E1 F1 (a_I + k3), B = E1 F1 (a_I + k1/6 + k2/3 + k3/3)
    NL_SDA = 6,         // A = F1 D(a_I + k3) -> C = F1 |D(a_I + k3)|^2
    NL_SDB = 7,         // A, B = F1 D(acc), C -> A = a' = D(acc) + k4/6 (real), C = F1 |a'|^2 unless nl_last
};
// Semi-implicit steps on 2D lattices keep one field, A, row-transformed between
// passes as F1 u / n1 (u = a_n, or u = D a_n on the way into a step):
enum SiOp {
    SI_ENTER = 0,       // A (real a) -> F1 a / n1
    SI_MUL = 1,         // A *= n1 E1 (sampling: the local terms of F1^-1 A first)
    SI_STEP = 2,        // A = F1 a_I / n1 -> a_I; m <- a_I + N(m)/2 three times; A = E1 F1 (2m - a_I) / n1
    SI_EXIT = 3         // A -> real F1^-1 A (sampling: its local terms)
};
enum ColMode {
    COL_PROPAGATE = 0,  // A, B -> F0^-1 E0 F0 (A, B)
    COL_SPECTRAL = 1,   // B: accumulate the kinetic energy only (no write)
    COL_FFT_FWD = 2,    // B <- F0 B (the middle transform of a 3D spectral sample)
    COL_SINGLE = 3,     // A -> F0^-1 E0 F0 A (the semi-implicit scheme's one field)
    COL_CONV = 4,       // C -> F0^-1 K2(k0, k1) F0 C (the non-local kernel, not separable)
    COL_FFT_BWD = 5     // B <- F0^-1 B (3D non-local term: the density's dimension-1 transform back)
};

template <typename R> struct Params2D {
    cx<R> *A;              // [npaths][N0][N1]
    cx<R> *B;              // scratch, same shape
    int64_t npaths;
    int n0, n1;
    const tw_t<R> *tw0, *tw1; // twiddles per dimension
    // separable exp(L dt/2) = E0(k0) E1(k1), each hi [n] then lo [n]; E0 carries
    // exp(c0 dt/2)/(n0 n1) and is applied by the column pass, E1 by the row
    // passes whose output feeds a column pass
    const cx<R> *E0, *E1;
    LocalTerm<R> lt;
    Sampling sm;
    int sample_slot;       // sample written by this pass (-1: none)
    uint64_t sg;           // global step index of the step this pass belongs to
    int *status;
    // 3D lattices reuse these passes: a row pass transforms the contiguous
    // dimension 2 (n0 := lines per path = N0*N1, n1 := N2, its line r is the
    // point pair (r / nmid, r % nmid) with nmid = N1); a column pass transforms
    // one strided dimension (n0 := its length, n1 := columns per slab, npaths :=
    // slabs).  kinner = N2 in the spectral pass along dimension 0 splits its
    // column index into (k1, k2); 0 for 2D.
    int ndim = 2;
    int nmid = 1;
    int kinner = 0;
    int si_op = 0;            // ROW_SI sub-operation (SiOp)
    int single_field = 0;     // TMA column pass: propagate A only (the semi-implicit scheme)
    double spec_scale = 1.0;  // COL_SPECTRAL: factor on |F0 B|^2 (B = F1 u / n1 needs n1^2)
    // 2D cosine (1) / sine (2) dimension 0 (generic column kernel): rows are
    // gathered in the even-odd order, E0 holds A and B0 B of
    // U_k = A_k V_k + B_k V_{n0-k} (hi [n0] then lo [n0] each)
    int basis0 = 0;
    const cx<R> *B0 = nullptr;
    // twiddles of the two-stage plan of dimension 0 (fft2.cuh), for the warp
    // column pass: entry (r-1) E + j holds w_n0^(r j), r < n0/E, j < E
    const tw_t<R> *tw0w = nullptr;
    // a cosine / sine dimension 1 of a 2D lattice (1 / 2; 0 Fourier) and the B
    // table of its pair step (hi[n1] | lo[n1]); E1 then holds the A table
    int basis1 = 0;
    const cx<R> *B1 = nullptr;
    // 3D spectral pass along dimension 0: the basis of dimension 2 (that of
    // dimension 1 in basis1); the column index splits as (k1, k2) by kinner
    int basis2 = 0;
    // complex64 TMA row pass: the paired twiddles of fftp_fwd / fftp_bwd (fft.cuh)
    // for the row dimension
    const tw_t<R> *tw1p = nullptr;
    // non-local term (2D, ROW_NL / COL_CONV): density / potential field C and the
    // real-space stage field D (same shape as A), the kernel K2 = khat / (n0 n1)
    // [n0][n1] in FFT order, the sub-operation and whether NL_SDB ends the run
    cx<R> *C = nullptr;
    cx<R> *D = nullptr;
    const cx<R> *K2 = nullptr;
    int nl_op = 0;
    int nl_last = 0;
};
template <typename R> cudaError_t launch_row_pass(int mode, const Params2D<R> &p, cudaStream_t s);
template <typename R> cudaError_t launch_col_pass(int mode, const Params2D<R> &p, cudaStream_t s);

// complex64 persistent TMA-pipelined variants (rk4ip_2d_tma.cu): the row pass
// for ROW_STAGE2/ROW_STEADY and the column pass for COL_PROPAGATE; `grid` is
// the number of SMs (the launchers place their persistent CTAs per SM).  Field
// bases must be 16-byte aligned; mapA/mapB describe A and B as [npaths*n0][n1]
// 8-byte elements with a COL_TMA_C x col_tma_box_rows(n0) box.
constexpr int COL_TMA_C = 8;   // columns per column-pass tile
bool tma_row_supported(int n1);   // row-pass line length
bool tma_col_supported(int n0);   // column length
size_t col_tma_box_rows(int n0);
cudaError_t launch_row_pass_tma(int mode, const Params2D<float> &p, int grid, cudaStream_t s);
cudaError_t launch_col_pass_tma(const Params2D<float> &p, const CUtensorMap &mapA, const CUtensorMap &mapB, int grid,
                                cudaStream_t s);

// complex64 column pass with warp-synchronous transforms (rk4ip_2d_warp.cu):
// COL_PROPAGATE on one or two fields over WARP_COL_C-column tiles with the
// two-stage plan of fft2.cuh (mapA/mapB: [npaths*n0][n1] 8-byte elements, box
// WARP_COL_C x warp_col_box_rows(n0), 64-byte swizzle).  `num_sms` sizes the
// persistent grid.
constexpr int WARP_COL_C = 8;
bool warp_col_supported(int n0, int64_t n1);      // column length and columns per slab
int warp_col_elems(int n0);                       // points per lane (E of the two-stage plan)
size_t warp_col_box_rows(int n0);
cudaError_t launch_col_pass_warp(const Params2D<float> &p, const CUtensorMap &mapA, const CUtensorMap &mapB,
                                 int num_sms, cudaStream_t s);

// --------------------------------------------------------------------------
// 1D adjoint: loss sum_p 1 - |<target|psi_N>|^2 and dL/dV (rk4ip_adjoint.cu)
// --------------------------------------------------------------------------
enum AdjPhase { ADJ_SEQUENTIAL = 0, ADJ_FORWARD = 1, ADJ_RECOMPUTE = 2, ADJ_REVERSE = 3 };
template <typename R> struct AdjParams {
    int phase;             // AdjPhase (see rk4ip_adjoint.cu)
    const cx<R> *psi0;     // [npaths][N]
    const cx<R> *target;   // [N]
    int64_t npaths;
    int64_t nsteps;
    int64_t K;             // checkpoint interval
    const cx<R> *Etab;     // hi [N] then lo [N]
    const tw_t<R> *tw;
    LocalTerm<R> lt;       // deterministic: noise off
    double dx;
    cx<R> *ckpt;           // [ceil(nsteps/K)][npaths][N]
    cx<R> *interm;         // [npaths][nsteps][4][N], or [npaths][K][4][N] (ADJ_SEQUENTIAL)
    cx<R> *final_state;    // [npaths][N] (the three-launch schedule)
    double *loss;          // accumulated (zeroed by the caller)
    double *dLdV;          // [nsteps][N], accumulated (zeroed by the caller)
    cx<R> *dLdpsi0;        // [npaths][N] or nullptr
    int *status = nullptr; // device error word (bounds-checking build)
    int64_t interm_steps = 0;  // steps held by interm (nsteps, or K)
};
template <typename R> cudaError_t launch_adjoint_1d(int n, int elems, const AdjParams<R> &p, cudaStream_t s);

// --------------------------------------------------------------------------
// Adaptive Cash-Karp 4(5) Runge-Kutta on 1D lattices (ark45_1d.cu): one CTA
// per path, each path with its own step size.
// --------------------------------------------------------------------------
enum { ST_STEP_LIMIT = 4 };   // a path used up its step attempts
template <typename R> struct AdaptiveParams {
    cx<R> *psi;            // [npaths][N] real space, in/out
    int64_t npaths;
    const tw_t<R> *tw;     // per-stage twiddles of the launch shape's radix plan
    cx<R> *kbuf;           // [npaths][6][N] stage derivatives (workspace)
    LocalTerm<R> lt;       // the static potential (noise off)
    double c0_re, c0_im, c2_re, c2_im;   // L(k) = c0 + c2 k^2
    double kscale;         // 2 pi / (xmax - xmin)
    double gnl;
    double t_end, tol, h0;
    int picture;           // 1: interaction picture, 0: explicit
    int64_t max_steps;     // step attempts per path
    int64_t *accepted, *rejected;   // [npaths] (device)
    int *status;
};
// points per thread of the launch shape for N (at least one warp per path)
int ark45_1d_elems(int n);
template <typename R> cudaError_t launch_ark45_1d(int n, const AdaptiveParams<R> &p, cudaStream_t s);

// --------------------------------------------------------------------------
// 0D: one thread per path (an ordinary SDE; D is a scalar factor).
// --------------------------------------------------------------------------
template <typename R> struct Params0D {
    cx<R> *psi;            // [npaths]
    int64_t npaths;
    int64_t nsteps;
    uint64_t step0;
    cx<R> Ehalf;           // exp(c0 dt/2)
    LocalTerm<R> lt;
    Sampling sm;
    int *status;
    int scheme = 0;        // 0 RK4IP, 1 semi-implicit midpoint
};
template <typename R> cudaError_t launch_rk4ip_0d(const Params0D<R> &p, cudaStream_t s);

// --------------------------------------------------------------------------
// Unfused comparison step (plain.cu): cuFFT transforms plus one elementwise
// kernel per operation, all fields in HBM between operations.
// --------------------------------------------------------------------------
template <typename R> struct PlainParams {
    cx<R> *a;              // [npaths][npts] real space, in/out
    cx<R> *aI, *k, *acc, *tmp; // work fields, same shape
    const cx<R> *E;        // exp(L(k) dt/2)/npts at every k (FFT order)
    int64_t npaths, npts;
    int ndim;
    int n[3];
    int64_t nsteps;
    uint64_t step0;
    LocalTerm<R> lt;
};
struct PlainPlan;
cudaError_t plain_plan_create(int ndim, const int *n, int64_t npaths, bool fp64, PlainPlan **out);
void plain_plan_destroy(PlainPlan *pl);
bool plain_plan_matches(const PlainPlan *pl, int ndim, const int *n, int64_t npaths, bool fp64);
template <typename R> cudaError_t run_plain(PlainPlan *pl, const PlainParams<R> &p, int num_sms, cudaStream_t s);

// Generator entry points (noise.cu).
cudaError_t launch_philox(const uint32_t *ctr, uint64_t seed, int64_t n, uint32_t *out, cudaStream_t s);
template <typename R>
cudaError_t launch_normals(uint64_t seed, int64_t npts, int64_t npaths, int64_t path_offset, uint32_t step,
                           void *out, cudaStream_t s);

// --------------------------------------------------------------------------
// Device helpers for the real-space term.
// --------------------------------------------------------------------------

// Per point and step: dt*(V + alpha xi_r) and the additive increment dt*sigma*xi_a.
template <typename R> struct PointTerm {
    R dtV;
    cx<R> na;
};

template <typename R>
__device__ __forceinline__ PointTerm<R> point_term(const LocalTerm<R> &lt, R Vraw, uint32_t j, uint32_t gpath,
                                                   uint32_t gstep) {
    PointTerm<R> pt;
    pt.dtV = lt.dt * Vraw;
    pt.na = mk<cx<R>>(R(0), R(0));
    if (lt.noise != NM_NONE) {
        // With substeps S the step's Wiener increment is the sum of those of S
        // steps S times shorter (fine global steps S n .. S n + S - 1): the same
        // Brownian path as a run with dt/S, normalised back to N(0, 1).
        cx<R> z = wiener_pair<R>(lt.key, j, gpath, gstep * (uint32_t)lt.substeps);
        if (lt.substeps > 1) {
            for (int i = 1; i < lt.substeps; ++i) {
                const cx<R> w = wiener_pair<R>(lt.key, j, gpath, gstep * (uint32_t)lt.substeps + (uint32_t)i);
                z.x += w.x;
                z.y += w.y;
            }
            const R r = R(1) / sqrt(R(lt.substeps));
            z.x *= r;
            z.y *= r;
        }
        if (lt.noise == NM_MUL_REAL) pt.dtV += lt.nscale * z.x;
        else if (lt.noise == NM_ADD_REAL) pt.na = mk<cx<R>>(lt.nscale * z.x, R(0));
        else pt.na = mk<cx<R>>(lt.nscale * z.x, lt.nscale * z.y);
    }
    return pt;
}

// N(u) = dt * (-i (V + alpha xi + g|u|^2) u + sigma xi_a)
template <typename R> __device__ __forceinline__ cx<R> apply_N(cx<R> u, const PointTerm<R> &pt, R gdt) {
    R dtpot = pt.dtV + gdt * cabs2(u);
    return mk<cx<R>>(dtpot * u.y + pt.na.x, -dtpot * u.x + pt.na.y);
}

// raw potential at flat point j (multi-index given) for global step gstep
template <typename R>
__device__ __forceinline__ R potential(const LocalTerm<R> &lt, int ndim, const int (&idx)[3], int64_t j,
                                       uint64_t gstep) {
    if (lt.pot == PM_HARMONIC) {
        R v = R(0);
        for (int d = 0; d < ndim; ++d) {
            const R x = lt.xmin[d] + R(idx[d]) * lt.dx[d];
            v += lt.hw2[d] * x * x;
        }
        return v;
    }
    if (lt.pot == PM_TABLE) {
        int64_t row = lt.V_nt > 1 ? (int64_t)gstep : 0;
        if (row >= lt.V_nt) row = lt.V_nt - 1;
        return XSDE_IN(row * lt.npts + j, lt.V_nt * lt.npts, lt.status) ? lt.V[row * lt.npts + j] : R(0);
    }
    return R(0);
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

}  // namespace xsde
