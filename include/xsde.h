/*
 * xsde.h -- C-ABI of the GB300 (sm_103a) RK4IP library.
 *
 * The library integrates (stochastic) PDEs of the form of XMDS2's
 * Eq. PDEBeforeIPTransform (Dennis, Hope & Johnsson, arXiv:1204.4255, Sec. 2.6),
 *
 *     d psi / dt = L[psi] + g(x, t, psi),
 *
 * on a periodic tensor-product Fourier lattice (Secs. 2.1-2.2) by the method of
 * lines (Sec. 2.5) with fourth-order Runge-Kutta in the interaction picture
 * (RK4IP, Sec. 2.6): the linear part L is solved exactly in Fourier space as
 * exp(L(k) dt/2) and g is evaluated in real space.  The closed equation family
 * accepted here covers the paper's NLS/GPE examples (Eq. NonlinearSchrodingerEquation,
 * Eq. NonlinearSchrodingerEquationDimensionless), the noisy trap of Example 6
 * (Sec. 3.6) and scalar SDEs:
 *
 *     L(k) = c0 + c2 |k|^2
 *     g    = -i (V(x, t) + g_nl |psi|^2 + alpha xi_r) psi + sigma xi_a
 *
 * with xi_r / xi_a real or complex spatial white Wiener noise (Sec. 2.5, in
 * Stratonovich form: one draw per step, point and path, fixed over the four
 * RK stages; variance 1/(dt dV) per step).
 *
 * Conventions
 *   - Lattice: x_j = xmin + j dx on [xmin, xmax), dx = (xmax - xmin)/N;
 *     k_j = 2 pi/(xmax - xmin) * (j < N/2 ? j : j - N).
 *   - Field layout: [path][n0][n1][n2] interleaved complex (re, im), the last
 *     grid dimension contiguous, paths outermost.  C64 = 2 x float,
 *     C128 = 2 x double.
 *   - Noise: Philox4x32-10 (Salmon et al., SC'11); the normal pair of global
 *     step n at point j of global path p comes from counter (j, p, n+1, 0) and
 *     key (seed_lo, seed_hi) through u = (x + 0.5) 2^-32 and Box-Muller:
 *     z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1).
 *     Real noise uses z0, complex noise (z0 + i z1)/sqrt(2).  Results are
 *     therefore independent of launch shape and of how paths are split.
 *
 * Errors: every call returns an xsde_status; on failure xsde_last_error()
 * returns a thread-local message.  No C++ exception crosses this boundary.
 * Device pointers are CUDA device (or managed) addresses on the current device;
 * `stream` arguments are cudaStream_t values passed as void*.
 */
#ifndef XSDE_H
#define XSDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XSDE_OK = 0,
    XSDE_EINVAL = 1,        /* invalid argument (checked on the host) */
    XSDE_ENOMEM = 2,        /* device allocation failed */
    XSDE_ECUDA = 3,         /* a CUDA runtime call failed */
    XSDE_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    XSDE_ENONFINITE = 5,    /* the field became NaN/Inf */
    XSDE_EUNSUPPORTED = 6,  /* valid but not implemented (size, dtype, combination) */
    XSDE_ELIMIT = 7,        /* an adaptive integration used up its step attempts */
    XSDE_EBOUNDS = 8        /* an index left its buffer (only the bounds-checking build,
                               libxsde_bounds.so, checks; the access was skipped) */
} xsde_status;

typedef enum { XSDE_C64 = 1, XSDE_C128 = 2 } xsde_dtype;

typedef enum {
    XSDE_POT_NONE = 0,
    XSDE_POT_HARMONIC = 1,  /* V = 1/2 sum_d omega_d^2 x_d^2 */
    XSDE_POT_TABLE = 2      /* V from a device table [V_nt][npts] */
} xsde_pot_kind;

typedef enum {
    XSDE_NOISE_NONE = 0,
    XSDE_NOISE_WIENER_REAL = 1,
    XSDE_NOISE_WIENER_COMPLEX = 2
} xsde_noise_kind;

typedef enum {
    XSDE_COUPLE_ADDITIVE = 0,        /* + sigma xi_a            (real or complex xi) */
    XSDE_COUPLE_MULTIPLICATIVE = 1   /* -i alpha xi_r psi       (real xi only) */
} xsde_noise_coupling;

enum {
    XSDE_MOM_NORM = 1,     /* per path: sum |psi|^2 dV */
    XSDE_MOM_ENERGY = 2,   /* per path: sum_k Re(i L(k)) |psi_k|^2 dV/N + sum_x (V|psi|^2 + g/2 |psi|^4) dV */
    XSDE_MOM_MOD2 = 4,     /* per point: mean over paths of |psi|^2 */
    XSDE_MOM_MOD4 = 8      /* per point: mean over paths of |psi|^4 */
};

typedef struct xsde_grid xsde_grid;
typedef struct xsde_vector xsde_vector;
typedef struct xsde_noise xsde_noise;
typedef struct xsde_problem xsde_problem;

/* Linear operator in Fourier space (Sec. 2.6): L(k) = c0 + c2 |k|^2. */
typedef struct {
    double c0_re, c0_im;
    double c2_re, c2_im;
} xsde_linear_op;

/* Local term in real space (Sec. 2.6, Eq. NonlinearSchrodingerEquation; noise
 * as in Example 6, Sec. 3.6).  V is a device pointer to a table of the
 * problem's real type (float for XSDE_C64, double for XSDE_C128) laid out
 * [V_nt][npts]: V_nt == 1 is a static table, otherwise row n is the potential
 * of global step n (piecewise constant over the step).  The table is borrowed:
 * the caller keeps it alive while integrations that use it are in flight. */
typedef struct {
    int32_t pot_kind;            /* xsde_pot_kind */
    double omega[3];             /* harmonic frequencies per dimension */
    const void *V;               /* device table, or NULL */
    int64_t V_nt;                /* rows of V */
    double g;                    /* g_nl */
    const xsde_noise *noise;     /* NULL: deterministic */
    int32_t coupling;            /* xsde_noise_coupling */
    double amplitude;            /* sigma (additive) or alpha (multiplicative) */
} xsde_nonlinear_op;

/* Sampling group (Sec. 3.1 "sampling", Sec. 3.6 averaged outputs): samples at
 * local steps 0, every, 2*every, ... <= nsteps of each xsde_integrate call. */
typedef struct {
    int32_t every;               /* 0: no sampling */
    int32_t which;               /* OR of XSDE_MOM_* */
} xsde_sampling;

/* ---- lattice (Secs. 2.1-2.2; dimensions of Example 2, Sec. 3.2) --------- */

/* ndim in 0..3 (0 = a single point: an ordinary SDE, dV = 1).  npts[d] is a
 * power of two in [16, 2048]; xmin[d] < xmax[d].  Arrays are read, not kept.
 * *out is owned by the caller (xsde_grid_destroy). */
int xsde_grid_create(int ndim, const int32_t *npts, const double *xmin, const double *xmax,
                     xsde_grid **out);
void xsde_grid_destroy(xsde_grid *grid);
/* number of lattice points (product of npts; 1 for ndim = 0) */
int64_t xsde_grid_points(const xsde_grid *grid);

/* Spectral basis per dimension (Sec. 2.1; Example 3, Sec. 3.3, halves a
 * reflection-symmetric problem's grid with the cosine basis).  A cosine (sine)
 * dimension of n points on (xmin, xmax) is cell-centred, x_j = xmin + (j+1/2)dx,
 * even (odd) about both ends, with modes cos / sin(k (x - xmin)) at
 * k = pi m/(xmax - xmin), m = 0..n-1 (cosine) or 1..n (sine): the DCT-II /
 * DST-II lattice.  The library evaluates these transforms with n-point FFTs
 * of the points taken in even-odd order (Makhoul's algorithm) and one pairing
 * of mode k with n-k.  basis: ndim entries of XSDE_BASIS_*, read during the
 * call; the default is all Fourier.  Set it before creating problems, fields
 * or noise from the grid (they copy it).  Runs on 1D lattices and on any
 * dimensions of 2D and 3D lattices (RK4IP; a cosine / sine last dimension runs
 * the generic row passes, and a 2D one takes its samples between chunks of
 * steps from the real-space field; 3D cosine / sine columns run the generic
 * column passes); the semi-implicit scheme on 2D and 3D lattices,
 * xsde_integrate_plain, xsde_integrate_adaptive, xsde_adjoint,
 * xsde_integrate_static_scratch and xsde_set_nonlocal report XSDE_EUNSUPPORTED
 * for such a problem.  A 1D cosine / sine problem has one launch shape
 * (xsde_kernel_variants reports 1); 2D keeps its four variants.  Energy
 * moments use the basis's Parseval weights.
 * Errors: XSDE_EINVAL for a NULL grid or basis, or an unknown value. */
#define XSDE_BASIS_FOURIER 0
#define XSDE_BASIS_COS 1
#define XSDE_BASIS_SIN 2
int xsde_grid_set_basis(xsde_grid *grid, const int32_t *basis);

/* ---- fields (Sec. 3.1 "vectors") ---------------------------------------- */

/* Allocate a device field of npaths x npts complex values (ncomp must be 1).
 * The library owns the memory (xsde_vector_free releases it). */
int xsde_vector_alloc(const xsde_grid *grid, xsde_dtype dtype, int ncomp, int64_t npaths,
                      xsde_vector **out);
/* Describe caller-owned device memory (e.g. a torch tensor) as a field.  The
 * memory is borrowed: it must stay alive and must not be used on other streams
 * while a call that uses it is in flight.  xsde_vector_free only frees the
 * descriptor. */
int xsde_vector_wrap(const xsde_grid *grid, xsde_dtype dtype, int ncomp, int64_t npaths,
                     void *dev_ptr, xsde_vector **out);
void *xsde_vector_data(const xsde_vector *vec);
void xsde_vector_free(xsde_vector *vec);

/* ---- noise (Sec. 2.5; noise_vector of Example 6, Sec. 3.6) -------------- */

/* A noise vector is not stored: it is (kind, seed) and regenerated from
 * Philox counters wherever it is needed. */
int xsde_noise_alloc(const xsde_grid *grid, xsde_noise_kind kind, uint64_t seed, xsde_noise **out);
void xsde_noise_free(xsde_noise *noise);

/* Raw generator words: out[i] = Philox4x32-10(counters[i], key = (seed_lo,
 * seed_hi)) for i < n.  counters and out are device arrays of n x 4 uint32,
 * 16-byte aligned, caller-owned.  Asynchronous on `stream`. */
int xsde_noise_philox(const uint32_t *counters, uint64_t seed, int64_t n, uint32_t *out, void *stream);

/* The standard normal pairs (z0, z1) that global step `step` draws for paths
 * path_offset .. path_offset+npaths-1 at points 0 .. npts-1, written to the
 * device array out[npaths][npts] of complex (z0, z1) in `dtype` (C64: FP32
 * Box-Muller, C128: FP64).  Asynchronous on `stream`. */
int xsde_noise_normals(const xsde_noise *noise, xsde_dtype dtype, int64_t npts, int64_t npaths,
                       int64_t path_offset, uint64_t step, void *out, void *stream);

/* ---- problem -------------------------------------------------------------- */

/* A problem binds a lattice, a precision and the operators; it owns the
 * device workspace (Fourier tables, one scratch field) that integration needs. */
int xsde_problem_create(const xsde_grid *grid, xsde_dtype dtype, xsde_problem **out);
void xsde_problem_destroy(xsde_problem *prob);

/* Set L (Fourier space) and g (real space).  Both structs are copied; the noise
 * handle and the V table are borrowed.  Multiplicative coupling needs real
 * noise; a potential table needs V != NULL and V_nt >= 1. */
int xsde_set_operators(xsde_problem *prob, const xsde_linear_op *L, const xsde_nonlinear_op *N);

/* The fixed-step scheme of xsde_integrate (and of batches): RK4IP (default),
 * or the semi-implicit midpoint step of Sec. 2.5's semi-implicit method in the
 * interaction picture of Sec. 2.6 -- a_I = D(a); m = a_I; m <- a_I + N(m)/2
 * three times; a <- D(2 m - a_I), with D = F^-1 exp(L dt/2) F and N = dt g with
 * the step's noise: deterministic order 2, strong order 1 (Stratonovich).  The
 * semi-implicit step runs on 0D to 3D Fourier lattices with one launch shape
 * (the problem reports one kernel variant while it is selected); on 2D and 3D
 * lattices it keeps one field and takes one row pass and one (2D) or two (3D)
 * column passes a step, the half-step factors of consecutive steps merged
 * into exp(L dt).  xsde_integrate on cosine / sine 2D lattices,
 * xsde_integrate_plain and xsde_adjoint report XSDE_EUNSUPPORTED for it. */
#define XSDE_SCHEME_RK4IP 0
#define XSDE_SCHEME_SEMI_IMPLICIT 1
int xsde_set_scheme(xsde_problem *prob, int32_t scheme);

/* Sample the same Brownian path at several step sizes (Sec. 2.5's strong
 * convergence test): with substeps S (1..65536, default 1) the noise of global
 * step n is built from the normals of the S finer steps S n .. S n + S - 1 --
 * their Wiener increments summed -- so a run with step dt and S substeps sees
 * the path of a run with step dt/S and substeps 1.  Global step indices times
 * S must stay below 2^32.  Applies to every integrating call of the problem. */
int xsde_set_noise_substeps(xsde_problem *prob, int32_t substeps);

/* Non-local pair potential (Example 5, Sec. 3.5: an interaction written as a
 * convolution, evaluated with FFTs).  g gains -i V_nl psi with
 *   V_nl = Re F^-1[ khat * F[|psi|^2] ],
 * F the unnormalised forward DFT of the lattice and F^-1 its inverse (with the
 * 1/npts), so that for khat = dx * DFT of a pair function f sampled at the
 * periodic offsets, V_nl(x) = sum_x' f(x - x') |psi(x')|^2 dx.  Every
 * evaluation of N in the step (four per RK4IP step) recomputes V_nl from its
 * own argument.  khat: HOST pointer to npts complex numbers, interleaved
 * (re, im) doubles in FFT order (index k at frequency k for k < npts/2, else
 * k - npts); read during the call and copied to the device in the problem's
 * precision.  NULL removes the term.  The call synchronises the device first,
 * so no integration in flight sees a half-written kernel.  Energy moments add
 * the pair energy 1/2 V_nl |psi|^2 dV.  1D, 2D and 3D Fourier lattices
 * (XSDE_EUNSUPPORTED on 0D lattices and cosine / sine lattices); on 2D
 * lattices khat is [n0][n1] and each N evaluation takes a density convolution
 * of its own (a row pass forming the density's row transform, a column pass
 * multiplying by khat, the evaluating row pass finishing the inverse), three
 * work fields of the field's size and twelve passes a step; on 3D lattices
 * khat is [n0][n1][n2] and each convolution adds the dimension-1 transforms of
 * the density (two more column passes).  Runs with RK4IP on one launch shape (xsde_kernel_variants
 * reports 1 while the term is set), and xsde_integrate with the semi-implicit scheme,
 * xsde_integrate_plain, xsde_integrate_adaptive and xsde_adjoint report
 * XSDE_EUNSUPPORTED while it is set.  Non-finite entries: XSDE_EINVAL. */
int xsde_set_nonlocal(xsde_problem *prob, const double *khat);

/* Diagnostics: dense fused-multiply-add throughput of the current device's
 * FP32 and FP64 pipes in TFLOP/s (8 independent FMA chains per thread, 64
 * warps per SM, timed with CUDA events after a warm-up launch; about 20 ms
 * each, synchronous, on the default stream).  These are the denominators of
 * the roofline fractions of arithmetic-bound kernels (the 1D whole-run kernel,
 * the complex128 passes).  Either pointer may be NULL to skip that pipe (not
 * both: XSDE_EINVAL); XSDE_ECUDA on a launch failure. */
int xsde_measure_fma_peaks(double *fp32_tflops, double *fp64_tflops);

/* Diagnostics: exercise the failure path of the bounded device-side waits
 * without a fault.  Launches on `stream` one CTA that waits, with the same
 * bounded mbarrier wait as the TMA pipelines, on a barrier that expects one
 * arrival nothing makes; after wait_ns nanoseconds (1e3..1e9, else
 * XSDE_EINVAL) it records the timeout in the problem's error word, so the next
 * xsde_synchronize reports XSDE_ETIMEOUT (and clears the word; the context
 * stays usable). */
int xsde_probe_wait_timeout(xsde_problem *prob, uint64_t wait_ns, void *stream);

/* Register a sampling group for the following xsde_integrate calls.
 * per_path  (device, FP64): [nsamp][npaths][2] = (norm, energy)  if NORM|ENERGY
 * per_point (device, FP64): [nsamp][npts][2]  = (mean |psi|^2, mean |psi|^4)
 *                                               if MOD2|MOD4
 * with nsamp = nsteps/every + 1.  Either pointer may be NULL when not needed;
 * entries that were not requested are left untouched.  Passing spec == NULL
 * or spec->every == 0 removes the sampling group. */
int xsde_moments(xsde_problem *prob, const xsde_sampling *spec, double *per_path, double *per_point);

/* Advance psi (all npaths paths, in place) by nsteps steps of size dt of the
 * problem's scheme (RK4IP unless xsde_set_scheme chose otherwise) on
 * `stream`, asynchronously.  Global path p of the noise counter is
 * path_offset + local path; the global step index is step_offset + local step
 * (this also selects the row of a time-dependent potential table).  Resuming
 * with step_offset = steps already taken reproduces an uninterrupted run.
 * npaths must equal the field's npaths.  Errors detected on the device are
 * reported by the next xsde_synchronize. */
int xsde_integrate(xsde_problem *prob, xsde_vector *psi, double dt, int64_t nsteps, int64_t npaths,
                   int64_t path_offset, uint64_t step_offset, void *stream);

/* As xsde_integrate for a field held in host memory: psi_in (host, npaths x
 * npts complex values of the problem's dtype, paths outermost) is copied to a
 * device field the problem owns (allocated on first use, grown when a larger
 * ensemble comes, freed with the problem), integrated, and copied back to
 * psi_out (host; may be psi_in) -- the host-to-device copy, every kernel and
 * the device-to-host copy in stream order on `stream`.  Returns once they are
 * issued; psi_out holds the result after the stream is synchronised
 * (xsde_synchronize).  Page-locked host buffers let the copies run
 * asynchronously; pageable ones make the copies synchronous with the host.
 * Arguments are checked as by xsde_integrate; a registered sampling group
 * fills its device buffers as there. */
int xsde_integrate_host(xsde_problem *prob, const void *psi_in, void *psi_out, int64_t npaths, double dt,
                        int64_t nsteps, int64_t path_offset, uint64_t step_offset, void *stream);

/* Gradient of a final-state fidelity through the discrete RK4IP scheme
 * (reverse mode through the step of Secs. 2.5-2.6; the workload of
 * Eq. InitialCondition driven by a space-time potential).  For the problem's
 * operators (deterministic; 1D lattice of 256..2048 points; the potential table,
 * if any, with one row per step and at least nsteps rows), the fields psi0
 * [npaths][N] and target [1][N] (device, borrowed, not modified):
 *   loss  (device, 1 double)          = sum_p 1 - |<target|psi_N>|^2, <a|b> = sum conj(a) b dx
 *   dLdV  (device, nsteps x N doubles) = dL/dV[n][j] with respect to the table
 *                                       entries (the potential of step n at point j)
 *   dLdpsi0 (device like psi0, or NULL) = lambda with dL = Re sum conj(lambda) dpsi0
 * psi_N is reached by nsteps steps of size dt.  States are checkpointed every
 * ckpt_every steps and each segment is recomputed once from its checkpoint (the
 * library owns that workspace).  When the stage inputs of all steps fit in
 * XSDE_ADJOINT_MAX_BYTES bytes of workspace (environment variable, default
 * 2 GiB) all segments are recomputed at once before the reverse sweep; else one
 * at a time during it, in a buffer of one segment.  Each path runs on one CTA
 * with 8 points per thread, or 4 when the problem's kernel variant is one of
 * the 1D 4- or 2-point shapes (xsde_set_kernel_variant) or, at the default
 * variant 0, when there are fewer paths than SMs.  Asynchronous on
 * `stream`. */
int xsde_adjoint(xsde_problem *prob, const xsde_vector *psi0, const xsde_vector *target, double dt, int64_t nsteps,
                 int32_t ckpt_every, double *loss, double *dLdV, void *dLdpsi0, void *stream);

/* ---- adaptive integration --------------------------------------------------- */

/* The adaptive fourth-fifth order Runge-Kutta of Sec. 2.5 (the Cash-Karp
 * embedded pair), in the interaction picture of Sec. 2.6 (picture = 1: the
 * linear part exp(L tau) applied exactly, the picture re-centred every step)
 * or on the explicit equation (picture = 0: L f evaluated spectrally at every
 * stage), the comparison of Fig. IPvsEX.  Each path advances from t = 0 to
 * t_end with its own step size: the step's error estimate
 * err = max_j |f5_j - f4_j| / max_j |f5_j| must be <= tol; the next step is
 * h clamp(0.9 (tol/err)^(1/5), 0.2, 5); a step that would pass t_end, or end
 * within 1e-12 t_end of it, ends on t_end; tol <= 0 takes fixed steps of h0. */
typedef struct {
    double t_end;       /* >= 0 */
    double tol;         /* relative error per step; <= 0: fixed steps of h0 */
    double h0;          /* first step, > 0 */
    int32_t picture;    /* 1: interaction picture, 0: explicit */
    int64_t max_steps;  /* step attempts per path (accepted + rejected), >= 1 */
} xsde_adaptive;

/* Integrate every path of psi (1D lattice of 64..2048 points, deterministic
 * operators with a static potential, no sampling group; else
 * XSDE_EUNSUPPORTED) as above, in place, asynchronously on `stream`.
 * accepted / rejected (device, int64 [npaths]) receive each path's step
 * counts.  A path that used up max_steps stops where it is and the next
 * xsde_synchronize reports XSDE_ELIMIT.  Each path runs on one CTA; the six
 * stage derivatives use the problem's workspace (6 fields). */
int xsde_integrate_adaptive(xsde_problem *prob, xsde_vector *psi, const xsde_adaptive *spec, int64_t *accepted,
                            int64_t *rejected, void *stream);

/* As xsde_integrate (1D-3D lattices, no sampling group), computed the plain
 * unfused way, for comparison with the fused passes: every transform is a
 * cuFFT call over all paths and every other operation of the step (exp(L dt/2)
 * from a table over all k, each N(u) = dt g(u), each Runge-Kutta combination)
 * is its own elementwise kernel with its operands in device memory.  The same
 * scheme (Secs. 2.5-2.6), noise counters and potential as xsde_integrate; the
 * results agree to rounding.  Allocates a cuFFT plan, four work fields and the
 * table on first use (or when the shape or dt changes) and waits for `stream`
 * then.  A registered sampling group, or a 0D lattice, reports
 * XSDE_EUNSUPPORTED. */
int xsde_integrate_plain(xsde_problem *prob, xsde_vector *psi, double dt, int64_t nsteps, int64_t npaths,
                         int64_t path_offset, uint64_t step_offset, void *stream);

/* As xsde_integrate, for 2D lattices, without allocating device memory.  The
 * paper has no counterpart; this call exists for callers that cannot call
 * cudaMalloc when they integrate (a fixed device-memory budget or a caller-owned
 * pool, real-time loops where an allocation would stall on a device-wide
 * synchronisation, hosts that give this library pointers but no heap growth).
 * Instead of the problem's own scratch field and Fourier tables it uses two
 * file-scope device arrays that every GPU loading the library holds until
 * process exit: a 16 MiB scratch field (npaths x points x element size must
 * not exceed 16 MiB, e.g. 8 paths of 512x512 complex64, else XSDE_EINVAL) and
 * 192 KiB of tables, rewritten by every call.  The call resolves the arrays'
 * device addresses the first time it runs on a device.  Every call copies its
 * tables from a host buffer with cudaMemcpyAsync and waits for `stream` before
 * it launches.  All calls
 * in the process share the arrays: calls that overlap on the GPU (other
 * streams, other threads) race and must not be issued.  The caller still
 * provides psi and any sampling buffers; the problem was created (and its
 * error word allocated) by xsde_problem_create.  Arguments are checked as by
 * xsde_integrate.  Other lattices, cosine / sine lattices, the semi-implicit
 * scheme and a non-local term report XSDE_EUNSUPPORTED. */
int xsde_integrate_static_scratch(xsde_problem *prob, xsde_vector *psi, double dt, int64_t nsteps,
                                  int64_t npaths, int64_t path_offset, uint64_t step_offset, void *stream);

/* Wait for `stream`, then report device-side errors of this problem's calls:
 * XSDE_ENONFINITE if a sampled field held NaN/Inf, XSDE_ETIMEOUT if a bounded
 * wait gave up, XSDE_ELIMIT if an adaptive path used up its step attempts,
 * XSDE_EBOUNDS if (in the bounds-checking build) a kernel computed an index
 * outside a field, table, sampling buffer or copy range.  Clears the device
 * error word. */
int xsde_synchronize(xsde_problem *prob, void *stream);

/* Kernel implementation for this problem, in [0, xsde_kernel_variants(prob)).
 * All variants compute the same scheme; they differ in launch shape:
 *   1D lattices (7 variants): variants 0-3 give each thread 8 points of a
 *     path (radix-8 stages) and one CTA the default number of paths (filling
 *     128 threads; one path for N >= 1024), a half (1), a quarter (2, at least
 *     one path) or twice (3, at most 256 threads) as many; variants 4 and 5
 *     give each thread 4 or 2 points (radix-4 or radix-2 stages, so a path
 *     spreads over more warps) with the default paths per CTA for that shape;
 *     variant 0 is compiled for 512 resident threads per SM in complex64 (at
 *     most 128 registers a thread, a few values spilled: more warps to hide
 *     the exchanges' latency) and with all its registers in complex128;
 *     variant 6 is variant 0 with the other choice; where a bound applies a
 *     variant repeats another;
 *   2D and 3D lattices (4 variants): 0 uses, in complex64, the persistent
 *     TMA-pipelined row pass (lines of 128..1024 points) and the column pass
 *     with warp-synchronous two-stage transforms (columns of 128..512 points,
 *     a multiple of 8 columns; else the TMA column pass), 1 forces the generic
 *     passes, 2 uses the TMA row passes and the generic column passes, 3 the
 *     TMA row and TMA column passes;
 *   0D lattices (1 variant).
 * Out-of-range variants report XSDE_EINVAL.  xsde_autotune picks one by
 * timing. */
int xsde_set_kernel_variant(xsde_problem *prob, int variant);
/* Number of kernel variants of the problem's lattice (0 if prob is NULL). */
int xsde_kernel_variants(const xsde_problem *prob);

/* ---- autotuning and batches ---------------------------------------------- */

/* Time every kernel variant of the problem (xsde_set_kernel_variant) over
 * nsteps >= 1 steps of size dt, on a device copy of psi (psi is read, not
 * modified; sampling and profiling are suspended meanwhile), and select the
 * fastest.  best (host, or NULL) receives its index; ms (host array of
 * xsde_kernel_variants(prob) doubles, or NULL) the best of three timed runs of
 * each variant.  With ms == NULL an earlier result for the same device,
 * lattice, precision and path count is reused: from this process, or from the
 * file named by the environment variable XSDE_AUTOTUNE_CACHE (text lines
 * "key variant", appended as results are found).  Allocates one field-sized
 * temporary and waits for `stream`. */
int xsde_autotune(xsde_problem *prob, const xsde_vector *psi, double dt, int64_t nsteps, int *best, double *ms,
                  void *stream);

/* A batch advances several independent problems together (the paper's paths
 * and separate simulations, Secs. 2.5 and 3): uneven lattices (0D..3D, any
 * sizes, either precision) in one replay of a CUDA graph of the members' pass
 * schedules.  The 0D / 1D members (one whole-run kernel each) are concurrent
 * branches; the 2D / 3D members, whose passes each occupy every SM, follow
 * them one after another.  Each member
 * names its own problem (its operators, sampling group, kernel variant and
 * scratch) and its field; the results equal those of one xsde_integrate per
 * member.  The paper has no batching call: its simulations run one at a time. */
typedef struct xsde_batch xsde_batch;
typedef struct {
    xsde_problem *prob;    /* borrowed; distinct across members */
    xsde_vector *psi;      /* borrowed; advanced in place; distinct across members */
    int64_t path_offset;   /* global path index of the field's path 0 */
} xsde_batch_member;

#define XSDE_BATCH_AUTOTUNE 1  /* xsde_autotune every member before the first replay */

/* Bind n >= 1 members (the array is copied; problems and fields must outlive
 * the batch and live on the current device).  Members that share a problem or
 * a field report XSDE_EINVAL. */
int xsde_batch_create(const xsde_batch_member *members, int n, int flags, xsde_batch **out);

/* Advance every member by nsteps steps of size dt from global step step_offset
 * (as xsde_integrate with npaths = the field's npaths), asynchronously on
 * `stream`.  The first call, and any call after a member's operators,
 * sampling group, kernel variant, field or workspace changed or with other
 * (dt, nsteps, step_offset), records the graph again (and, with
 * XSDE_BATCH_AUTOTUNE, the first call tunes the members); otherwise the call
 * is one graph launch.  Recording waits for `stream`.  Device-side errors are
 * reported per member by xsde_synchronize(member problem, stream). */
int xsde_batch_integrate(xsde_batch *batch, double dt, int64_t nsteps, uint64_t step_offset, void *stream);

/* Wait for the device, then free the batch (not its members). */
void xsde_batch_destroy(xsde_batch *batch);

/* ---- launch profiling ------------------------------------------------------ */

/* Kernel kinds reported by xsde_profile_report, in this order:
 * rk4ip_0d, rk4ip_1d, row_prologue, row_stage2, row_steady, row_epilogue,
 * row_fft_only, col_propagate, col_spectral, row_nonlocal, col_convolve (see
 * xsde_kernel_name). */
#define XSDE_KERNEL_KINDS 11

/* Start (enable != 0) or stop recording a CUDA event pair around every kernel
 * launch of this problem, on the launch stream; resets the totals.  Separately,
 * with the environment variable XSDE_NVTX=1 every such launch is also wrapped
 * in an NVTX range named after its kind (for timeline tools). */
int xsde_profile(xsde_problem *prob, int enable);
/* Wait for the recorded events and return, per kernel kind, the summed device
 * time in ms and the number of launches since xsde_profile (host arrays of
 * XSDE_KERNEL_KINDS entries). */
int xsde_profile_report(xsde_problem *prob, double *total_ms, int64_t *launches);
/* Name of kernel kind `kind` ("" if out of range). */
const char *xsde_kernel_name(int kind);

/* ---- errors --------------------------------------------------------------- */

/* Message of the last failed call on this thread ("" if none). */
const char *xsde_last_error(void);
/* Library version string. */
const char *xsde_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XSDE_H */
