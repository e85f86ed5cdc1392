/*
 * xsde_oracle.c -- plain FP64 CPU oracle for the RK4IP method-of-lines step of
 * XMDS2 (Dennis, Hope & Johnsson, arXiv:1204.4255).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the GPU library.
 *
 * What it computes (one function per paper item):
 *   - separable complex FFT on a periodic tensor-product lattice: Sec. 2.2
 *     (fast spatial-to-spectral transforms) and the Fourier basis of Sec. 2.1;
 *     textbook iterative radix-2 Cooley-Tukey with bit reversal.  Forward is
 *     unnormalised (sign -1), inverse is scaled by 1/N (sign +1).
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
 *     SC'11) and Box-Muller normals: the Wiener increments of Sec. 2.5.
 *   - RK4 in the interaction picture: Sec. 2.5 (method of lines, classical RK4)
 *     combined with Sec. 2.6 (Eqs. PDEBeforeIPTransform/PDEAfterIPTransform),
 *     with the picture re-centred every step so that only exp(L dt/2) is needed.
 *   - norm and energy by equal-weight quadrature (Sec. 2.4, Fourier case) and
 *     per-point ensemble moments over paths (Sec. 2.5, multiple paths).
 *   - the cosine and sine bases of Sec. 2.1 (Example 3 halves a symmetric
 *     problem's grid with the cosine transform): per dimension, the DCT-II /
 *     DST-II written out as sums of cosines / sines and their exact inverses.
 *
 * Conventions (the readings where the paper is silent):
 *   - lattice x_j = xmin + j*dx on [xmin, xmax), dx = (xmax-xmin)/N;
 *     k_j = 2*pi/(xmax-xmin) * (j < N/2 ? j : j-N);
 *   - cosine / sine dimensions: cell-centred points x_j = xmin + (j + 1/2) dx
 *     (even / odd reflection about both ends), modes cos(k_n (x - xmin)) with
 *     k_n = pi n/(xmax-xmin), n = 0..N-1, and sin(k_n (x - xmin)) with
 *     k_n = pi (n+1)/(xmax-xmin); forward transforms unnormalised,
 *     X_n = sum_j x_j cos(pi n (j+1/2)/N) (sin(pi (n+1) (j+1/2)/N)), and the
 *     inverses exact (so D = C^-1 exp(L dt/2) C);
 *   - array layout [path][n0][n1][n2], the last grid dimension contiguous;
 *   - L(k) = c0 + c2*|k|^2;
 *     g(x,t,psi) = -i*(V(x,t) + gnl*|psi|^2 + alpha*xi_r)*psi + sigma*xi_a,
 *     with xi_r a real and xi_a a real or complex spatial white noise,
 *     <xi(x) xi(x')> = delta/(dt*dV) per step, held fixed over the 4 stages
 *     (Stratonovich limit, Sec. 2.5);
 *   - noise of global step n, point j, path p: Philox counter
 *     (j, p, n+1, 0), key (seed & 0xffffffff, seed >> 32); uniforms
 *     u = (x + 0.5) * 2^-32; z0 = sqrt(-2 ln u0) cos(2 pi u1),
 *     z1 = sqrt(-2 ln u0) sin(2 pi u1).  Real noise uses z0, complex noise
 *     (z0 + i z1)/sqrt(2).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define TWO_PI 6.283185307179586476925286766559
#define PI 3.1415926535897932384626433832795

typedef struct {
    int32_t ndim;      /* 0 (a single point: an ordinary SDE) .. 3 */
    int32_t n[3];      /* points per dimension, powers of two */
    double xmin[3];
    double xmax[3];
    int32_t basis[3];  /* per dimension: 0 Fourier (periodic), 1 cosine (even), 2 sine (odd) */
} oracle_grid;

enum { BASIS_FOURIER = 0, BASIS_COS = 1, BASIS_SIN = 2 };

typedef struct {
    double c0_re, c0_im;   /* L(k) = c0 + c2 |k|^2 */
    double c2_re, c2_im;
    double gnl;            /* nonlinear coefficient g */
    double noise_amp;      /* sigma (additive) or alpha (multiplicative) */
    double omega[3];       /* harmonic trap V = 1/2 sum omega_i^2 x_i^2 */
    const double *V;       /* potential table [V_nt][npts] */
    int64_t V_nt;          /* rows of the table: 1 = static, else one per step */
    uint64_t seed;
    int32_t pot_kind;      /* 0 none, 1 harmonic, 2 table */
    int32_t noise_kind;    /* 0 none, 1 additive real, 2 additive complex,
                              3 multiplicative real */
    int32_t substeps;      /* noise of step n from the finer steps S n .. S n + S - 1
                              (the same Brownian path as steps S times shorter);
                              values below 1 mean 1 */
    int32_t scheme;        /* 0: RK4IP; 1: semi-implicit midpoint in the interaction
                              picture (see oracle_rk4ip) */
    const double *knl;     /* non-local kernel in Fourier space, [npts] complex in FFT
                              order, or NULL: g gains -i V_nl psi with
                              V_nl = iFFT(knl * FFT(|psi|^2)) (Example 5's convolution) */
} oracle_ops;

enum { POT_NONE = 0, POT_HARMONIC = 1, POT_TABLE = 2 };
enum { NOISE_NONE = 0, NOISE_ADD_REAL = 1, NOISE_ADD_COMPLEX = 2, NOISE_MUL_REAL = 3 };

/* ------------------------------------------------------------------------- */
/* Lattice                                                                   */
/* ------------------------------------------------------------------------- */

static int64_t grid_points(const oracle_grid *g)
{
    int64_t n = 1;
    for (int d = 0; d < g->ndim; d++) n *= g->n[d];
    return n;
}

static double grid_dx(const oracle_grid *g, int d)
{
    return (g->xmax[d] - g->xmin[d]) / g->n[d];
}

static double grid_dV(const oracle_grid *g)
{
    double v = 1.0;
    for (int d = 0; d < g->ndim; d++) v *= grid_dx(g, d);
    return v;
}

/* multi-index of flat point index j (last dimension fastest) */
static void unflatten(const oracle_grid *g, int64_t j, int idx[3])
{
    for (int d = g->ndim - 1; d >= 0; d--) {
        idx[d] = (int)(j % g->n[d]);
        j /= g->n[d];
    }
}

static double coord_x(const oracle_grid *g, int d, int i)
{
    double off = g->basis[d] == BASIS_FOURIER ? 0.0 : 0.5;
    return g->xmin[d] + (i + off) * grid_dx(g, d);
}

static double coord_k(const oracle_grid *g, int d, int i)
{
    int n = g->n[d];
    if (g->basis[d] == BASIS_COS) return PI * i / (g->xmax[d] - g->xmin[d]);
    if (g->basis[d] == BASIS_SIN) return PI * (i + 1) / (g->xmax[d] - g->xmin[d]);
    int m = (i < n / 2) ? i : i - n;
    return TWO_PI / (g->xmax[d] - g->xmin[d]) * m;
}

/* weight of spectral point j in Parseval's sum: sum_x |u|^2 = sum_k w_k |U_k|^2 / npts.
   Fourier modes weigh 1; a cosine or sine dimension weighs 2, except its mode that
   has no partner (the constant cosine, the highest sine) */
static double spectral_weight(const oracle_grid *g, int64_t j)
{
    int idx[3];
    unflatten(g, j, idx);
    double w = 1.0;
    for (int d = 0; d < g->ndim; d++) {
        if (g->basis[d] == BASIS_COS && idx[d] != 0) w *= 2.0;
        if (g->basis[d] == BASIS_SIN && idx[d] != g->n[d] - 1) w *= 2.0;
    }
    return w;
}

static double ksq_at(const oracle_grid *g, int64_t j)
{
    int idx[3];
    unflatten(g, j, idx);
    double s = 0.0;
    for (int d = 0; d < g->ndim; d++) {
        double k = coord_k(g, d, idx[d]);
        s += k * k;
    }
    return s;
}

/* ------------------------------------------------------------------------- */
/* FFT: iterative radix-2 Cooley-Tukey on one contiguous line                */
/* ------------------------------------------------------------------------- */

static void fft_line(cplx *x, int n, int sign)
{
    /* bit-reversal reordering */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    /* butterflies of doubling length; each twiddle evaluated directly */
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; k++) {
            double ang = sign * TWO_PI * k / len;
            cplx w = cos(ang) + I * sin(ang);
            for (int i = 0; i < n; i += len) {
                cplx u = x[i + k];
                cplx v = x[i + k + half] * w;
                x[i + k] = u + v;
                x[i + k + half] = u - v;
            }
        }
    }
    if (sign > 0) {
        for (int i = 0; i < n; i++) x[i] /= n;
    }
}

/* DCT-II (sign -1) of one line, or its inverse (sign +1), as plain sums */
static void dct_line(cplx *x, int n, int sign)
{
    cplx *y = malloc(sizeof(cplx) * n);
    for (int a = 0; a < n; a++) {
        cplx acc = 0.0;
        if (sign < 0) {           /* X_a = sum_j x_j cos(pi a (j + 1/2) / n) */
            for (int j = 0; j < n; j++) acc += x[j] * cos(PI * a * (j + 0.5) / n);
        } else {                  /* x_a = (X_0 + 2 sum_{m>0} X_m cos(pi m (a + 1/2) / n)) / n */
            acc = x[0];
            for (int m = 1; m < n; m++) acc += 2.0 * x[m] * cos(PI * m * (a + 0.5) / n);
            acc /= n;
        }
        y[a] = acc;
    }
    memcpy(x, y, sizeof(cplx) * n);
    free(y);
}

/* DST-II (sign -1) of one line, or its inverse (sign +1), as plain sums */
static void dst_line(cplx *x, int n, int sign)
{
    cplx *y = malloc(sizeof(cplx) * n);
    for (int a = 0; a < n; a++) {
        cplx acc = 0.0;
        if (sign < 0) {           /* X_a = sum_j x_j sin(pi (a + 1) (j + 1/2) / n) */
            for (int j = 0; j < n; j++) acc += x[j] * sin(PI * (a + 1) * (j + 0.5) / n);
        } else {                  /* x_a = (sum_{m<n-1} 2 X_m sin(..) + X_{n-1} sin(..)) / n */
            for (int m = 0; m < n; m++)
                acc += (m == n - 1 ? 1.0 : 2.0) * x[m] * sin(PI * (m + 1) * (a + 0.5) / n);
            acc /= n;
        }
        y[a] = acc;
    }
    memcpy(x, y, sizeof(cplx) * n);
    free(y);
}

/* Transform every line of every dimension of nbatch stacked arrays. */
static void fft_nd(cplx *data, const oracle_grid *g, int64_t nbatch, int sign)
{
    int64_t npts = grid_points(g);
    for (int d = 0; d < g->ndim; d++) {
        int n = g->n[d];
        int64_t stride = 1;
        for (int e = d + 1; e < g->ndim; e++) stride *= g->n[e];
        int64_t outer = npts / (stride * n);
        int64_t nlines = nbatch * outer * stride;
        #pragma omp parallel for schedule(static)
        for (int64_t line = 0; line < nlines; line++) {
            int64_t b = line / (outer * stride);
            int64_t r = line % (outer * stride);
            int64_t o = r / stride, s = r % stride;
            cplx *base = data + b * npts + o * stride * n + s;
            cplx *tmp = malloc(sizeof(cplx) * n);
            for (int i = 0; i < n; i++) tmp[i] = base[i * stride];
            if (g->basis[d] == BASIS_COS) dct_line(tmp, n, sign);
            else if (g->basis[d] == BASIS_SIN) dst_line(tmp, n, sign);
            else fft_line(tmp, n, sign);
            for (int i = 0; i < n; i++) base[i * stride] = tmp[i];
            free(tmp);
        }
    }
}

void oracle_fft(double *data, const oracle_grid *g, int64_t nbatch, int32_t sign)
{
    fft_nd((cplx *)data, g, nbatch, sign);
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 and Box-Muller                                              */
/* ------------------------------------------------------------------------- */

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t r0 = hi1 ^ c[1] ^ k[0];
    uint32_t r1 = lo1;
    uint32_t r2 = hi0 ^ c[3] ^ k[1];
    uint32_t r3 = lo0;
    c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int round = 0; round < 10; round++) {
        if (round > 0) {           /* Weyl-sequence key schedule */
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    for (int i = 0; i < 4; i++) out[i] = c[i];
}

void oracle_philox_batch(const uint32_t *ctr, const uint32_t *key, int64_t m, uint32_t *out)
{
    for (int64_t i = 0; i < m; i++) oracle_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

static double uniform_open(uint32_t x)
{
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

/* the normal pair (z0, z1) that step `step` draws at (point j, path p) */
static void wiener_pair(uint64_t seed, int64_t j, int64_t p, int64_t step, double z[2])
{
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)p, (uint32_t)(step + 1), 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    oracle_philox4x32_10(ctr, key, x);
    double u0 = uniform_open(x[0]), u1 = uniform_open(x[1]);
    double r = sqrt(-2.0 * log(u0));
    z[0] = r * cos(TWO_PI * u1);
    z[1] = r * sin(TWO_PI * u1);
}

void oracle_wiener_normals(uint64_t seed, int64_t npts, int64_t npaths, int64_t path0,
                           int64_t step, double *z)
{
    for (int64_t p = 0; p < npaths; p++)
        for (int64_t j = 0; j < npts; j++)
            wiener_pair(seed, j, path0 + p, step, z + 2 * (p * npts + j));
}

/* ------------------------------------------------------------------------- */
/* The equation: L(k) in Fourier space, g(x, t, psi) in real space           */
/* ------------------------------------------------------------------------- */

static double potential_at(const oracle_grid *g, const oracle_ops *ops, int64_t j, int64_t step)
{
    if (ops->pot_kind == POT_HARMONIC) {
        int idx[3];
        unflatten(g, j, idx);
        double v = 0.0;
        for (int d = 0; d < g->ndim; d++) {
            double x = coord_x(g, d, idx[d]);
            v += 0.5 * ops->omega[d] * ops->omega[d] * x * x;
        }
        return v;
    }
    if (ops->pot_kind == POT_TABLE) {
        int64_t row = (ops->V_nt > 1) ? step : 0;
        if (row >= ops->V_nt) row = ops->V_nt - 1;
        return ops->V[row * grid_points(g) + j];
    }
    return 0.0;
}

/* exp(L(k) dt/2) on every point of the lattice */
static void half_step_factors(const oracle_grid *g, const oracle_ops *ops, double dt, cplx *E)
{
    cplx c0 = ops->c0_re + I * ops->c0_im;
    cplx c2 = ops->c2_re + I * ops->c2_im;
    int64_t npts = grid_points(g);
    for (int64_t j = 0; j < npts; j++) E[j] = cexp((c0 + c2 * ksq_at(g, j)) * (0.5 * dt));
}

/* D(u) = iFFT( exp(L dt/2) FFT(u) ), applied to every path */
static void apply_D(cplx *u, const cplx *E, const oracle_grid *g, int64_t npaths)
{
    int64_t npts = grid_points(g);
    fft_nd(u, g, npaths, -1);
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npaths * npts; i++) u[i] *= E[i % npts];
    fft_nd(u, g, npaths, +1);
}

typedef struct {
    double *Vrow;   /* potential of this step [npts] */
    cplx *xi_a;     /* additive noise of this step [npaths][npts] (or NULL) */
    double *xi_m;   /* multiplicative noise of this step [npaths][npts] (or NULL) */
    const oracle_grid *g;   /* the lattice, for the non-local term */
} step_inputs;

/* V_nl of one path: the circular convolution of |u|^2 with the kernel whose
   DFT is ops->knl, evaluated as iFFT(knl * FFT(|u|^2)) (Example 5) */
static void nonlocal_potential(const oracle_grid *g, const oracle_ops *ops, const cplx *u, double *vnl)
{
    int64_t npts = grid_points(g);
    const cplx *knl = (const cplx *)ops->knl;
    cplx *rho = malloc(sizeof(cplx) * npts);
    for (int64_t j = 0; j < npts; j++) rho[j] = creal(u[j]) * creal(u[j]) + cimag(u[j]) * cimag(u[j]);
    fft_nd(rho, g, 1, -1);
    for (int64_t j = 0; j < npts; j++) rho[j] *= knl[j];
    fft_nd(rho, g, 1, +1);
    for (int64_t j = 0; j < npts; j++) vnl[j] = creal(rho[j]);
    free(rho);
}

/* the non-local potential of every path, for the tests: u, out [npaths][npts] */
void oracle_nonlocal_potential(const oracle_grid *g, const oracle_ops *ops, const double *u, int64_t npaths,
                               double *out)
{
    int64_t npts = grid_points(g);
    for (int64_t p = 0; p < npaths; p++) nonlocal_potential(g, ops, (const cplx *)u + p * npts, out + p * npts);
}

/* out = N(u) = dt * g(x, t_n, u) for every path */
static void nonlinear(cplx *out, const cplx *u, const oracle_ops *ops, const step_inputs *in,
                      int64_t npts, int64_t npaths, double dt)
{
    double *vnl = NULL;
    if (ops->knl && in->g) {
        vnl = malloc(sizeof(double) * npaths * npts);
        for (int64_t p = 0; p < npaths; p++) nonlocal_potential(in->g, ops, u + p * npts, vnl + p * npts);
    }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npaths * npts; i++) {
        int64_t j = i % npts;
        double mod2 = creal(u[i]) * creal(u[i]) + cimag(u[i]) * cimag(u[i]);
        double pot = in->Vrow[j] + ops->gnl * mod2;
        if (vnl) pot += vnl[i];
        if (in->xi_m) pot += ops->noise_amp * in->xi_m[i];
        cplx gval = -I * pot * u[i];
        if (in->xi_a) gval += ops->noise_amp * in->xi_a[i];
        out[i] = dt * gval;
    }
    free(vnl);
}

static void fill_step_inputs(step_inputs *in, const oracle_grid *g, const oracle_ops *ops,
                             int64_t npaths, int64_t path0, int64_t step, double dt)
{
    int64_t npts = grid_points(g);
    in->g = g;
    for (int64_t j = 0; j < npts; j++) in->Vrow[j] = potential_at(g, ops, j, step);
    if (ops->noise_kind == NOISE_NONE) return;
    double scale = 1.0 / sqrt(dt * grid_dV(g));   /* white noise per step: var 1/(dt dV) */
    const int64_t S = ops->substeps > 1 ? ops->substeps : 1;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < npaths * npts; i++) {
        int64_t p = i / npts, j = i % npts;
        /* the Wiener increment of the step is the sum of the S finer steps'
           increments: z = (sum of their standard normals) / sqrt(S) */
        double z[2] = {0.0, 0.0};
        for (int64_t f = 0; f < S; f++) {
            double zf[2];
            wiener_pair(ops->seed, j, path0 + p, S * step + f, zf);
            z[0] += zf[0];
            z[1] += zf[1];
        }
        z[0] /= sqrt((double)S);
        z[1] /= sqrt((double)S);
        if (ops->noise_kind == NOISE_ADD_REAL) in->xi_a[i] = scale * z[0];
        else if (ops->noise_kind == NOISE_ADD_COMPLEX) in->xi_a[i] = scale * (z[0] + I * z[1]) / sqrt(2.0);
        else in->xi_m[i] = scale * z[0];
    }
}

/* ------------------------------------------------------------------------- */
/* Observables                                                               */
/* ------------------------------------------------------------------------- */

/* per path: norm = sum |psi|^2 dV and
 * energy = sum_k Re(i L(k)) |psi_k|^2 dV / N + sum_x (V |psi|^2 + g/2 |psi|^4) dV */
void oracle_observables(const oracle_grid *g, const oracle_ops *ops, const double *psi_in,
                        int64_t npaths, int64_t step, double *out)
{
    const cplx *psi = (const cplx *)psi_in;
    int64_t npts = grid_points(g);
    double dV = grid_dV(g);
    cplx *spec = malloc(sizeof(cplx) * npaths * npts);
    double *vnl = ops->knl ? malloc(sizeof(double) * npts) : NULL;
    memcpy(spec, psi, sizeof(cplx) * npaths * npts);
    fft_nd(spec, g, npaths, -1);
    for (int64_t p = 0; p < npaths; p++) {
        double norm = 0.0, e_lin = 0.0, e_loc = 0.0;
        if (vnl) nonlocal_potential(g, ops, psi + p * npts, vnl);
        for (int64_t j = 0; j < npts; j++) {
            cplx u = psi[p * npts + j];
            double m2 = creal(u) * creal(u) + cimag(u) * cimag(u);
            norm += m2 * dV;
            e_loc += (potential_at(g, ops, j, step) * m2 + 0.5 * ops->gnl * m2 * m2) * dV;
            if (vnl) e_loc += 0.5 * vnl[j] * m2 * dV;   /* pair interaction energy */
            cplx s = spec[p * npts + j];
            double s2 = creal(s) * creal(s) + cimag(s) * cimag(s);
            double hk = -ops->c0_im - ops->c2_im * ksq_at(g, j);    /* Re(i L(k)) */
            e_lin += hk * spectral_weight(g, j) * s2 * dV / npts;
        }
        out[2 * p] = norm;
        out[2 * p + 1] = e_lin + e_loc;
    }
    free(spec);
    free(vnl);
}

/* ------------------------------------------------------------------------- */
/* RK4 in the interaction picture                                            */
/* ------------------------------------------------------------------------- */

/*
 * RK4IP, one step from t_n to t_n + dt for all paths (a is real-space psi, updated):
 *   a_I = D(a)
 *   k1  = D(N(a))
 *   k2  = N(a_I + k1/2)
 *   k3  = N(a_I + k2/2)
 *   k4  = N(D(a_I + k3))
 *   a  <- D(a_I + k1/6 + k2/3 + k3/3) + k4/6
 * with D = exp(L dt/2) applied in Fourier space and N = dt*g in real space.
 * ops->scheme = 1 takes the semi-implicit midpoint step instead:
 *   a_I = D(a);  m = a_I;  m <- a_I + N(m)/2 (three times);  a <- D(2 m - a_I).
 */

/*
 * Integrate nsteps RK4IP steps.  psi: [npaths][npts] complex (in/out).
 * Paths are the global paths path0 .. path0+npaths-1; steps are the global
 * steps step0 .. step0+nsteps-1 (the noise and the potential table row follow
 * the global indices).  If sample_every > 0, samples are taken at local steps
 * 0, S, 2S, ... <= nsteps:
 *   per_path  [nsamp][npaths][2] = (norm, energy)
 *   per_point [nsamp][npts][2]   = (mean |psi|^2, mean |psi|^4) over the paths
 * Returns 0, or -1 on an invalid argument.
 */
int oracle_rk4ip(const oracle_grid *g, const oracle_ops *ops, double *psi_in, int64_t npaths,
                 int64_t path0, double dt, int64_t nsteps, int64_t step0, int32_t sample_every,
                 double *per_path, double *per_point)
{
    if (g->ndim < 0 || g->ndim > 3 || npaths < 1 || nsteps < 0) return -1;
    for (int d = 0; d < g->ndim; d++) {
        if (g->n[d] < 1 || (g->n[d] & (g->n[d] - 1))) return -1;
        if (g->basis[d] < BASIS_FOURIER || g->basis[d] > BASIS_SIN) return -1;
        if (ops->knl && g->basis[d] != BASIS_FOURIER) return -1;   /* a circular convolution */
    }
    if (ops->pot_kind == POT_TABLE && ops->V_nt > 1 && step0 + nsteps > ops->V_nt) return -1;

    cplx *a = (cplx *)psi_in;
    int64_t npts = grid_points(g), m = npaths * npts;
    cplx *E = malloc(sizeof(cplx) * npts);
    cplx *aI = malloc(sizeof(cplx) * m), *k1 = malloc(sizeof(cplx) * m);
    cplx *k2 = malloc(sizeof(cplx) * m), *k3 = malloc(sizeof(cplx) * m);
    cplx *k4 = malloc(sizeof(cplx) * m), *tmp = malloc(sizeof(cplx) * m);
    step_inputs in;
    in.Vrow = malloc(sizeof(double) * npts);
    in.xi_a = (ops->noise_kind == NOISE_ADD_REAL || ops->noise_kind == NOISE_ADD_COMPLEX)
                  ? malloc(sizeof(cplx) * m) : NULL;
    in.xi_m = (ops->noise_kind == NOISE_MUL_REAL) ? malloc(sizeof(double) * m) : NULL;
    double *obs = malloc(sizeof(double) * 2 * npaths);

    half_step_factors(g, ops, dt, E);

    int64_t sample = 0;
    for (int64_t n = 0; n <= nsteps; n++) {
        if (sample_every > 0 && n % sample_every == 0) {
            if (per_path) {
                oracle_observables(g, ops, psi_in, npaths, step0 + n, obs);
                memcpy(per_path + sample * npaths * 2, obs, sizeof(double) * 2 * npaths);
            }
            if (per_point) {
                double *pp = per_point + sample * npts * 2;
                for (int64_t j = 0; j < npts; j++) {
                    double s2 = 0.0, s4 = 0.0;
                    for (int64_t p = 0; p < npaths; p++) {
                        cplx u = a[p * npts + j];
                        double m2 = creal(u) * creal(u) + cimag(u) * cimag(u);
                        s2 += m2;
                        s4 += m2 * m2;
                    }
                    pp[2 * j] = s2 / npaths;
                    pp[2 * j + 1] = s4 / npaths;
                }
            }
            sample++;
        }
        if (n == nsteps) break;

        fill_step_inputs(&in, g, ops, npaths, path0, step0 + n, dt);

        if (ops->scheme == 1) {
            /* semi-implicit midpoint in the interaction picture (Sec. 2.5's
               semi-implicit method, Werner & Drummond 1997, with Sec. 2.6):
               a_I = D(a); m <- a_I + N(m)/2 three times from m = a_I;
               a <- D(2 m - a_I) */
            memcpy(aI, a, sizeof(cplx) * m);
            apply_D(aI, E, g, npaths);
            memcpy(tmp, aI, sizeof(cplx) * m);
            for (int it = 0; it < 3; it++) {
                nonlinear(k1, tmp, ops, &in, npts, npaths, dt);
                for (int64_t i = 0; i < m; i++) tmp[i] = aI[i] + 0.5 * k1[i];
            }
            for (int64_t i = 0; i < m; i++) tmp[i] = 2.0 * tmp[i] - aI[i];
            apply_D(tmp, E, g, npaths);
            memcpy(a, tmp, sizeof(cplx) * m);
            continue;
        }

        /* a_I = D(a) */
        memcpy(aI, a, sizeof(cplx) * m);
        apply_D(aI, E, g, npaths);
        /* k1 = D(N(a)) */
        nonlinear(k1, a, ops, &in, npts, npaths, dt);
        apply_D(k1, E, g, npaths);
        /* k2 = N(a_I + k1/2) */
        for (int64_t i = 0; i < m; i++) tmp[i] = aI[i] + 0.5 * k1[i];
        nonlinear(k2, tmp, ops, &in, npts, npaths, dt);
        /* k3 = N(a_I + k2/2) */
        for (int64_t i = 0; i < m; i++) tmp[i] = aI[i] + 0.5 * k2[i];
        nonlinear(k3, tmp, ops, &in, npts, npaths, dt);
        /* k4 = N(D(a_I + k3)) */
        for (int64_t i = 0; i < m; i++) tmp[i] = aI[i] + k3[i];
        apply_D(tmp, E, g, npaths);
        nonlinear(k4, tmp, ops, &in, npts, npaths, dt);
        /* a <- D(a_I + k1/6 + k2/3 + k3/3) + k4/6 */
        for (int64_t i = 0; i < m; i++) tmp[i] = aI[i] + k1[i] / 6.0 + k2[i] / 3.0 + k3[i] / 3.0;
        apply_D(tmp, E, g, npaths);
        for (int64_t i = 0; i < m; i++) a[i] = tmp[i] + k4[i] / 6.0;
    }

    free(E); free(aI); free(k1); free(k2); free(k3); free(k4); free(tmp);
    free(in.Vrow); free(in.xi_a); free(in.xi_m); free(obs);
    return 0;
}

/* number of samples oracle_rk4ip writes for (nsteps, sample_every) */
int64_t oracle_num_samples(int64_t nsteps, int32_t sample_every)
{
    return sample_every > 0 ? nsteps / sample_every + 1 : 0;
}

/* threads used by the OpenMP loops over lines and points (1 = serial) */
void oracle_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int32_t oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the discrete RK4IP step (discretise-then-differentiate)        */
/* ------------------------------------------------------------------------- */
/*
 * Fields are real vectors (Re, Im) with the inner product <u, v> = Re sum conj(u) v.
 * For N(u) = dt (-i (V + g|u|^2) u) (no noise), the tangent is
 *   dN = A du + B conj(du),   A = -i dt (V + 2 g |u|^2),  B = -i dt g u^2,
 * and its adjoint maps a cotangent mu to conj(A) mu + B conj(mu).  D = F^-1 E F
 * has adjoint F^-1 conj(E) F.  dN/dV_j = -i dt u_j, so a stage with cotangent
 * mu adds Re(conj(mu_j) (-i dt u_j)) to dL/dV_j.
 */

static void apply_Dadj(cplx *u, const cplx *E, const oracle_grid *g, int64_t npaths)
{
    int64_t npts = grid_points(g);
    fft_nd(u, g, npaths, -1);
    for (int64_t i = 0; i < npaths * npts; i++) u[i] *= conj(E[i % npts]);
    fft_nd(u, g, npaths, +1);
}

/* one path: the forward step's intermediates from its input a */
typedef struct {
    cplx *a, *aI, *k1, *w2, *k2, *w3, *k3, *Du1, *acc;
} step_state;

static void step_forward_store(step_state *s, const cplx *E, const oracle_grid *g, const oracle_ops *ops,
                               const step_inputs *in, double dt, cplx *out)
{
    int64_t m = grid_points(g);
    memcpy(s->aI, s->a, sizeof(cplx) * m);
    apply_D(s->aI, E, g, 1);
    nonlinear(s->k1, s->a, ops, in, m, 1, dt);
    apply_D(s->k1, E, g, 1);
    for (int64_t i = 0; i < m; i++) s->w2[i] = s->aI[i] + 0.5 * s->k1[i];
    nonlinear(s->k2, s->w2, ops, in, m, 1, dt);
    for (int64_t i = 0; i < m; i++) s->w3[i] = s->aI[i] + 0.5 * s->k2[i];
    nonlinear(s->k3, s->w3, ops, in, m, 1, dt);
    for (int64_t i = 0; i < m; i++) s->Du1[i] = s->aI[i] + s->k3[i];
    apply_D(s->Du1, E, g, 1);
    for (int64_t i = 0; i < m; i++) s->acc[i] = s->aI[i] + s->k1[i] / 6.0 + s->k2[i] / 3.0 + s->k3[i] / 3.0;
    apply_D(s->acc, E, g, 1);
    if (out) {
        cplx *k4 = malloc(sizeof(cplx) * m);
        nonlinear(k4, s->Du1, ops, in, m, 1, dt);
        for (int64_t i = 0; i < m; i++) out[i] = s->acc[i] + k4[i] / 6.0;
        free(k4);
    }
}

/* cotangent of N's input for cotangent mu of its output, at input u */
static cplx adj_N(cplx u, cplx mu, double Vj, double g, double dt)
{
    double m2 = creal(u) * creal(u) + cimag(u) * cimag(u);
    cplx A = -I * dt * (Vj + 2.0 * g * m2);
    cplx B = -I * dt * g * u * u;
    return conj(A) * mu + B * conj(mu);
}

static double dV_term(cplx mu, cplx u, double dt)
{
    return creal(conj(mu) * (-I * dt * u));
}

/* Reverse of one step: lam (cotangent of a_{n+1}) -> cotangent of a_n; adds dL/dV_n to gV. */
static void step_adjoint(const step_state *s, const cplx *E, const oracle_grid *g, const oracle_ops *ops,
                         const step_inputs *in, double dt, const cplx *lam_next, cplx *lam, double *gV)
{
    int64_t m = grid_points(g);
    cplx *l_acc = malloc(sizeof(cplx) * m), *l_u1 = malloc(sizeof(cplx) * m);
    cplx *l_k1 = malloc(sizeof(cplx) * m), *l_aI = malloc(sizeof(cplx) * m);
    /* a' = D acc + k4/6, k4 = N(Du1) */
    for (int64_t i = 0; i < m; i++) {
        cplx l_k4 = lam_next[i] / 6.0;
        l_acc[i] = lam_next[i];
        l_u1[i] = adj_N(s->Du1[i], l_k4, in->Vrow[i], ops->gnl, dt);
        gV[i] += dV_term(l_k4, s->Du1[i], dt);
    }
    apply_Dadj(l_acc, E, g, 1);     /* acc = a_I + k1/6 + k2/3 + k3/3 */
    apply_Dadj(l_u1, E, g, 1);      /* Du1 = D(a_I + k3) */
    for (int64_t i = 0; i < m; i++) {
        cplx la = l_acc[i], lu = l_u1[i];
        cplx l_aIi = la + lu;
        cplx l_k3 = la / 3.0 + lu;
        cplx l_w3 = adj_N(s->w3[i], l_k3, in->Vrow[i], ops->gnl, dt);     /* k3 = N(w3), w3 = a_I + k2/2 */
        gV[i] += dV_term(l_k3, s->w3[i], dt);
        l_aIi += l_w3;
        cplx l_k2 = la / 3.0 + 0.5 * l_w3;
        cplx l_w2 = adj_N(s->w2[i], l_k2, in->Vrow[i], ops->gnl, dt);     /* k2 = N(w2), w2 = a_I + k1/2 */
        gV[i] += dV_term(l_k2, s->w2[i], dt);
        l_aIi += l_w2;
        l_k1[i] = la / 6.0 + 0.5 * l_w2;
        l_aI[i] = l_aIi;
    }
    apply_Dadj(l_k1, E, g, 1);      /* k1 = D N(a) */
    apply_Dadj(l_aI, E, g, 1);      /* a_I = D a */
    for (int64_t i = 0; i < m; i++) {
        lam[i] = adj_N(s->a[i], l_k1[i], in->Vrow[i], ops->gnl, dt) + l_aI[i];
        gV[i] += dV_term(l_k1[i], s->a[i], dt);
    }
    free(l_acc); free(l_u1); free(l_k1); free(l_aI);
}

static void state_alloc(step_state *s, int64_t m)
{
    cplx **f[] = {&s->a, &s->aI, &s->k1, &s->w2, &s->k2, &s->w3, &s->k3, &s->Du1, &s->acc};
    for (int i = 0; i < 9; i++) *f[i] = malloc(sizeof(cplx) * m);
}

static void state_free(step_state *s)
{
    cplx *f[] = {s->a, s->aI, s->k1, s->w2, s->k2, s->w3, s->k3, s->Du1, s->acc};
    for (int i = 0; i < 9; i++) free(f[i]);
}

/*
 * Loss L = sum over paths of 1 - |<target|psi_N>|^2, <a|b> = sum conj(a) b dV,
 * after nsteps RK4IP steps (deterministic; potential from ops, a table with one
 * row per step or static).  Writes the loss, dL/dV[n][j] (w.r.t. the table
 * entries of step n; zero rows are written when the potential is not a table)
 * and dL/dpsi0 as the cotangent lam with dL = Re sum conj(lam) dpsi0.
 * All states are stored (no checkpointing: this is the plain reference).
 */
int oracle_adjoint(const oracle_grid *g, const oracle_ops *ops, const double *psi0_in, int64_t npaths,
                   const double *target_in, double dt, int64_t nsteps, double *loss, double *dLdV,
                   double *dLdpsi0)
{
    if (ops->noise_kind != NOISE_NONE || nsteps < 1 || ops->knl) return -1;
    if (ops->pot_kind == POT_TABLE && ops->V_nt > 1 && nsteps > ops->V_nt) return -1;
    int64_t m = grid_points(g);
    double dV = grid_dV(g);
    const cplx *target = (const cplx *)target_in;
    cplx *E = malloc(sizeof(cplx) * m);
    half_step_factors(g, ops, dt, E);
    cplx *states = malloc(sizeof(cplx) * m * (nsteps + 1));
    step_state s;
    state_alloc(&s, m);
    step_inputs in = {malloc(sizeof(double) * m), NULL, NULL};
    cplx *lam = malloc(sizeof(cplx) * m), *lam_prev = malloc(sizeof(cplx) * m);
    memset(dLdV, 0, sizeof(double) * nsteps * m);
    *loss = 0.0;
    for (int64_t p = 0; p < npaths; p++) {
        memcpy(states, psi0_in + 2 * p * m, sizeof(cplx) * m);
        for (int64_t n = 0; n < nsteps; n++) {
            fill_step_inputs(&in, g, ops, 1, p, n, dt);
            memcpy(s.a, states + n * m, sizeof(cplx) * m);
            step_forward_store(&s, E, g, ops, &in, dt, states + (n + 1) * m);
        }
        cplx c = 0.0;
        for (int64_t j = 0; j < m; j++) c += conj(target[j]) * states[nsteps * m + j] * dV;
        *loss += 1.0 - (creal(c) * creal(c) + cimag(c) * cimag(c));
        for (int64_t j = 0; j < m; j++) lam[j] = -2.0 * c * target[j] * dV;
        for (int64_t n = nsteps - 1; n >= 0; n--) {
            fill_step_inputs(&in, g, ops, 1, p, n, dt);
            memcpy(s.a, states + n * m, sizeof(cplx) * m);
            step_forward_store(&s, E, g, ops, &in, dt, NULL);
            step_adjoint(&s, E, g, ops, &in, dt, lam, lam_prev, dLdV + n * m);
            memcpy(lam, lam_prev, sizeof(cplx) * m);
        }
        if (dLdpsi0) memcpy(dLdpsi0 + 2 * p * m, lam, sizeof(cplx) * m);
    }
    state_free(&s);
    free(E); free(states); free(in.Vrow); free(lam); free(lam_prev);
    return 0;
}

/*
 * One step's tangent (forward mode) and adjoint, for the transpose test:
 *   tangent: da_out = J_a da + J_V dV   (dV a perturbation of this step's potential)
 *   adjoint: lam_out = J_a^T lam, gV = J_V^T lam
 */
int oracle_step_tangent(const oracle_grid *g, const oracle_ops *ops, const double *a_in, const double *da_in,
                        const double *dVrow, int64_t step, double dt, double *da_out)
{
    if (ops->knl) return -1;
    int64_t m = grid_points(g);
    const cplx *a = (const cplx *)a_in, *da = (const cplx *)da_in;
    cplx *E = malloc(sizeof(cplx) * m);
    half_step_factors(g, ops, dt, E);
    step_inputs in = {malloc(sizeof(double) * m), NULL, NULL};
    fill_step_inputs(&in, g, ops, 1, 0, step, dt);
    step_state s;
    state_alloc(&s, m);
    memcpy(s.a, a, sizeof(cplx) * m);
    step_forward_store(&s, E, g, ops, &in, dt, NULL);
    /* tangent of N at u: A du + B conj(du) + (-i dt u) dV */
    #define TAN_N(u, du, j) (-I * dt * (in.Vrow[j] + 2.0 * ops->gnl * (creal(u) * creal(u) + cimag(u) * cimag(u))) * (du) \
                             - I * dt * ops->gnl * (u) * (u) * conj(du) - I * dt * (u) * dVrow[j])
    cplx *t_aI = malloc(sizeof(cplx) * m), *t_k1 = malloc(sizeof(cplx) * m), *t_k2 = malloc(sizeof(cplx) * m);
    cplx *t_k3 = malloc(sizeof(cplx) * m), *t_u1 = malloc(sizeof(cplx) * m), *t_acc = malloc(sizeof(cplx) * m);
    memcpy(t_aI, da, sizeof(cplx) * m);
    apply_D(t_aI, E, g, 1);
    for (int64_t j = 0; j < m; j++) t_k1[j] = TAN_N(a[j], da[j], j);
    apply_D(t_k1, E, g, 1);
    for (int64_t j = 0; j < m; j++) t_k2[j] = TAN_N(s.w2[j], t_aI[j] + 0.5 * t_k1[j], j);
    for (int64_t j = 0; j < m; j++) t_k3[j] = TAN_N(s.w3[j], t_aI[j] + 0.5 * t_k2[j], j);
    for (int64_t j = 0; j < m; j++) t_u1[j] = t_aI[j] + t_k3[j];
    apply_D(t_u1, E, g, 1);
    for (int64_t j = 0; j < m; j++) t_acc[j] = t_aI[j] + t_k1[j] / 6.0 + t_k2[j] / 3.0 + t_k3[j] / 3.0;
    apply_D(t_acc, E, g, 1);
    cplx *out = (cplx *)da_out;
    for (int64_t j = 0; j < m; j++) out[j] = t_acc[j] + TAN_N(s.Du1[j], t_u1[j], j) / 6.0;
    #undef TAN_N
    free(t_aI); free(t_k1); free(t_k2); free(t_k3); free(t_u1); free(t_acc);
    state_free(&s);
    free(E); free(in.Vrow);
    return 0;
}

int oracle_step_adjoint(const oracle_grid *g, const oracle_ops *ops, const double *a_in, const double *lam_in,
                        int64_t step, double dt, double *lam_out, double *gV)
{
    if (ops->knl) return -1;
    int64_t m = grid_points(g);
    cplx *E = malloc(sizeof(cplx) * m);
    half_step_factors(g, ops, dt, E);
    step_inputs in = {malloc(sizeof(double) * m), NULL, NULL};
    fill_step_inputs(&in, g, ops, 1, 0, step, dt);
    step_state s;
    state_alloc(&s, m);
    memcpy(s.a, a_in, sizeof(cplx) * m);
    step_forward_store(&s, E, g, ops, &in, dt, NULL);
    memset(gV, 0, sizeof(double) * m);
    step_adjoint(&s, E, g, ops, &in, dt, (const cplx *)lam_in, (cplx *)lam_out, gV);
    state_free(&s);
    free(E); free(in.Vrow);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adaptive fourth-fifth order Runge-Kutta (Sec. 2.5: the Cash-Karp embedded */
/* pair), in the interaction picture of Sec. 2.6 or on the explicit equation */
/* ------------------------------------------------------------------------- */
/*
 * Deterministic equation df/dt = L f + g(f), g(f) = -i (V(x) + gnl |f|^2) f.
 * One step of size h from t:
 *   interaction picture (picture = 1): with f~(s) = exp(-L s) f(t + s), the
 *     stages are k_i = h exp(-L c_i h) g(exp(L c_i h) Y_i), Y_i = f + sum_j a_ij k_j,
 *     the fifth-order result is f~5 = f + sum_i b5_i k_i and the step ends with
 *     f(t + h) = exp(L h) f~5 (the picture is re-centred at every step);
 *   explicit (picture = 0): k_i = h (L Y_i + g(Y_i)), f(t + h) = f + sum_i b5_i k_i.
 * Error estimate e = sum_i (b5_i - b4_i) k_i; err = max_j |e_j| / max_j |f5_j|
 * (f5 the fifth-order result of the step, in the frame the stages use).  A
 * step is accepted when err <= tol; either way the next size is
 * h * clamp(0.9 (tol/err)^(1/5), 0.2, 5) (5 when err = 0), and a step that
 * would pass t_end, or end within 1e-12 t_end of it, is set to end on t_end.  tol <= 0 selects fixed steps of
 * h0 (never rejected; the last one shortened).
 */

/* Cash & Karp (1990), ACM TOMS 16, 201: nodes, coupling and the two weights */
static const double CK_C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double CK_A[6][5] = {
    {0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
static const double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double CK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0,
                                1.0 / 4.0};

/* the tableau, for the tests: c[6], a[6][5] row-major, b5[6], b4[6] */
void oracle_cash_karp(double *c, double *a, double *b5, double *b4)
{
    for (int i = 0; i < 6; i++) {
        c[i] = CK_C[i];
        b5[i] = CK_B5[i];
        b4[i] = CK_B4[i];
        for (int j = 0; j < 5; j++) a[i * 5 + j] = CK_A[i][j];
    }
}

/* exp(L(k) tau) times u, in place (u in real space on entry and exit) */
static void propagate(cplx *u, const oracle_grid *g, const oracle_ops *ops, double tau)
{
    if (tau == 0.0) return;
    cplx c0 = ops->c0_re + I * ops->c0_im;
    cplx c2 = ops->c2_re + I * ops->c2_im;
    int64_t npts = grid_points(g);
    fft_nd(u, g, 1, -1);
    for (int64_t j = 0; j < npts; j++) u[j] *= cexp((c0 + c2 * ksq_at(g, j)) * tau);
    fft_nd(u, g, 1, +1);
}

/* out = L u = iFFT(L(k) FFT(u)) */
static void apply_L(cplx *out, const cplx *u, const oracle_grid *g, const oracle_ops *ops)
{
    cplx c0 = ops->c0_re + I * ops->c0_im;
    cplx c2 = ops->c2_re + I * ops->c2_im;
    int64_t npts = grid_points(g);
    memcpy(out, u, (size_t)npts * sizeof(cplx));
    fft_nd(out, g, 1, -1);
    for (int64_t j = 0; j < npts; j++) out[j] *= c0 + c2 * ksq_at(g, j);
    fft_nd(out, g, 1, +1);
}

/* g(u) = -i (V + gnl |u|^2) u */
static void g_det(cplx *out, const cplx *u, const double *Vrow, const oracle_ops *ops, int64_t npts)
{
    for (int64_t j = 0; j < npts; j++) {
        double mod2 = creal(u[j]) * creal(u[j]) + cimag(u[j]) * cimag(u[j]);
        out[j] = -I * (Vrow[j] + ops->gnl * mod2) * u[j];
    }
}

/* one path from t = 0 to t_end; returns 0, or 1 when max_steps attempts ran out */
static int ark45_path(const oracle_grid *g, const oracle_ops *ops, const double *Vrow, cplx *y, double t_end,
                      double tol, double h0, int picture, int64_t max_steps, int64_t *accepted,
                      int64_t *rejected)
{
    int64_t npts = grid_points(g);
    cplx *k = malloc((size_t)6 * npts * sizeof(cplx));
    cplx *Y = malloc((size_t)npts * sizeof(cplx));
    cplx *v = malloc((size_t)npts * sizeof(cplx));
    cplx *Lv = malloc((size_t)npts * sizeof(cplx));
    double t = 0.0, h = h0;
    int64_t acc = 0, rej = 0;
    int rc = 0;
    while (t < t_end) {
        if (acc + rej >= max_steps) { rc = 1; break; }
        /* end exactly on t_end (a step within 1e-12 t_end of it is stretched) */
        if (t + h > t_end || t_end - (t + h) <= 1e-12 * t_end) h = t_end - t;
        for (int i = 0; i < 6; i++) {
            cplx *ki = k + (size_t)i * npts;
            for (int64_t j = 0; j < npts; j++) {
                cplx s = y[j];
                for (int m = 0; m < i; m++) s += CK_A[i][m] * k[(size_t)m * npts + j];
                Y[j] = s;
            }
            if (picture) {
                const double tau = CK_C[i] * h;
                propagate(Y, g, ops, tau);
                g_det(v, Y, Vrow, ops, npts);
                propagate(v, g, ops, -tau);
                for (int64_t j = 0; j < npts; j++) ki[j] = h * v[j];
            } else {
                g_det(v, Y, Vrow, ops, npts);
                apply_L(Lv, Y, g, ops);
                for (int64_t j = 0; j < npts; j++) ki[j] = h * (Lv[j] + v[j]);
            }
        }
        double emax = 0.0, ymax = 0.0;
        for (int64_t j = 0; j < npts; j++) {
            cplx y5 = y[j], e = 0.0;
            for (int i = 0; i < 6; i++) {
                y5 += CK_B5[i] * k[(size_t)i * npts + j];
                e += (CK_B5[i] - CK_B4[i]) * k[(size_t)i * npts + j];
            }
            Y[j] = y5;
            if (cabs(e) > emax) emax = cabs(e);
            if (cabs(y5) > ymax) ymax = cabs(y5);
        }
        const double err = ymax > 0.0 ? emax / ymax : 0.0;
        if (tol <= 0.0 || err <= tol) {
            t += h;
            memcpy(y, Y, (size_t)npts * sizeof(cplx));
            if (picture) propagate(y, g, ops, h);
            acc++;
        } else {
            rej++;
        }
        if (tol > 0.0) {
            double fac = err > 0.0 ? 0.9 * pow(tol / err, 0.2) : 5.0;
            if (fac < 0.2) fac = 0.2;
            if (fac > 5.0) fac = 5.0;
            h *= fac;
        } else {
            h = h0;
        }
    }
    *accepted = acc;
    *rejected = rej;
    free(k);
    free(Y);
    free(v);
    free(Lv);
    return rc;
}

/* Adaptive integration of every path to t_end (see the block comment above).
 * Deterministic problems with a static potential only.  Returns 0, -1 for
 * arguments it does not accept, 1 if some path ran out of max_steps attempts
 * (its field is then the state it reached). */
int oracle_ark45(const oracle_grid *g, const oracle_ops *ops, double *psi_in, int64_t npaths, double t_end,
                 double tol, double h0, int32_t picture, int64_t max_steps, int64_t *accepted,
                 int64_t *rejected)
{
    if (ops->noise_kind != NOISE_NONE || ops->knl || (ops->pot_kind == POT_TABLE && ops->V_nt != 1)) return -1;
    if (!(t_end >= 0.0) || !(h0 > 0.0) || g->ndim < 1) return -1;
    int64_t npts = grid_points(g);
    double *Vrow = malloc((size_t)npts * sizeof(double));
    for (int64_t j = 0; j < npts; j++) Vrow[j] = potential_at(g, ops, j, 0);
    cplx *psi = (cplx *)psi_in;
    int rc = 0;
    #pragma omp parallel for schedule(dynamic) reduction(| : rc)
    for (int64_t p = 0; p < npaths; p++)
        rc |= ark45_path(g, ops, Vrow, psi + p * npts, t_end, tol, h0, picture, max_steps, accepted + p,
                         rejected + p);
    free(Vrow);
    return rc;
}
