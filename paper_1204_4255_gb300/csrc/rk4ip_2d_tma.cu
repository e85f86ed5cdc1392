// rk4ip_2d_tma.cu -- the complex64 2D passes as persistent, TMA-pipelined kernels.
//
// Same arithmetic as rk4ip_2d.cu (XMDS2 Sec. 2.6: exp(L dt/2) in Fourier space,
// the real-space RK4 stages in between; Sec. 2.2: separable transforms), laid
// out for sm_103a: one CTA per SM walks a list of 64 KB work items; three
// shared-memory stages hold the item being transformed and the next two, which
// the tensor-memory-access unit is already copying in (cp.async.bulk, completion
// on an mbarrier with a byte count).  Each FFT runs in place in the staged tile
// and the result leaves through a bulk store, so the SM never waits on a global
// load while it computes and no register holds data in flight.
//   row item    : ROWS consecutive lines of A and of B (2 x 32 KB, 1D bulk copies)
//   column item : an 8-column x n0-row tile of A or of B (32 KB, 2D tensor copies);
//                 two CTAs per SM, so one CTA's exchanges overlap the other's arithmetic
// Row exchanges use an XOR swizzle within each line (conflict-free for n1 = 512);
// column tiles are naturally conflict-free (a half-warp touches two whole 64-byte rows).
#include <type_traits>

#include "fft.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace xsde {
namespace {

using V = float2;
using TW = float4;
constexpr int NST = 3;                        // shared-memory stages
constexpr uint64_t kWaitNs = 2000000000ull;    // give up on a copy after 2 s

// slot of element i of a line during row exchanges
struct SwizzledLine {
    __device__ __forceinline__ int operator()(int i) const { return i ^ ((i >> 4) & 7) ^ (((i >> 6) & 1) << 3); }
};

template <int T>
__device__ __forceinline__ void line_sum2(double (&v)[2], int t, int line, double *scratch) {
    if constexpr (T <= 32) {
#pragma unroll
        for (int o = T / 2; o > 0; o >>= 1)
#pragma unroll
            for (int i = 0; i < 2; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    } else {
        constexpr int W = T / 32;
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

// on a copy that never lands: record it and drain what this CTA has in flight
__device__ void give_up(int *status, uint64_t *bars, const uint32_t *parity_next) {
    if (threadIdx.x == 0) {
        atomicOr(status, ST_TIMEOUT);
        for (int s = 0; s < NST; ++s) mbar_wait(bars + s, parity_next[s], kWaitNs);
        bulk_wait<0>();
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Row pass
// ---------------------------------------------------------------------------
template <int N1> struct RowTma {
    static constexpr int E = 8;
    static constexpr int T = N1 / E;
    static constexpr int ROWS = 4096 / N1;               // 2 x ROWS x N1 x 8 B = 64 KB per item
    static constexpr int THREADS = ROWS * T;              // 512
    static constexpr size_t ITEM = (size_t)2 * ROWS * N1 * sizeof(V);
    static constexpr size_t SCRATCH = (size_t)ROWS * (T / 32 + 1) * 2 * sizeof(double);
    static constexpr size_t SMEM = NST * ITEM + (size_t)N1 * sizeof(TW) + (size_t)2 * N1 * sizeof(V) + SCRATCH +
                                   NST * sizeof(uint64_t);
};

// SAMPLE: this pass writes a sample (ROW_STEADY only); NOISE: the problem has
// Wiener noise.  Both are template flags so the common pass carries neither the
// sampling code nor the generator.
template <int N1, int MODE, bool SAMPLE, bool NOISE>
__global__ void __launch_bounds__(RowTma<N1>::THREADS, 1) row_pass_tma_kernel(const Params2D<float> p) {
    using Cfg = RowTma<N1>;
    constexpr int E = Cfg::E, T = Cfg::T, ROWS = Cfg::ROWS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *bufs = reinterpret_cast<V *>(smem_raw);
    TW *tw_s = reinterpret_cast<TW *>(smem_raw + NST * Cfg::ITEM);
    V *e1_s = reinterpret_cast<V *>(tw_s + N1);
    double *scratch = reinterpret_cast<double *>(e1_s + 2 * N1);
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(scratch) + Cfg::SCRATCH);

    const int tid = threadIdx.x;
    const int line = tid / T, t = tid - line * T;
    const int64_t nitems = p.npaths * (int64_t)p.n0 / ROWS;
    const int64_t mine = nitems > blockIdx.x ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const size_t vec_bytes = (size_t)ROWS * N1 * sizeof(V);

    // the paired twiddles as (c, s) and (c eps, s eps) halves in tw_s's N1 entries
    float2 *tw_hi = reinterpret_cast<float2 *>(tw_s), *tw_lo = tw_hi + N1;
    stage_paired(tw_hi, tw_lo, p.tw1p, N1, tid, blockDim.x);
    for (int i = tid; i < 2 * N1; i += blockDim.x) e1_s[i] = p.E1[i];
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(bars + s, 1);
        fence_barrier_init();
    }
    __syncthreads();
    // the tables above are constants; the fields are the previous pass's output
    grid_launch_dependents();
    grid_dependency_wait();

    auto issue_load = [&](int64_t k) {   // item k of this CTA into stage k % NST
        const int s = (int)(k % NST);
        const int64_t row0 = (blockIdx.x + k * gridDim.x) * ROWS;
        V *dst = bufs + (size_t)s * 2 * ROWS * N1;
        // (bounds-checking build: a copy past the fields is skipped, the stage
        // completes without bytes)
        if (!XSDE_IN(row0 + ROWS - 1, p.npaths * (int64_t)p.n0, p.status)) {
            mbar_arrive(bars + s);
            return;
        }
        mbar_arrive_expect_tx(bars + s, (uint32_t)(2 * vec_bytes));
        bulk_load(dst, p.A + row0 * N1, (uint32_t)vec_bytes, bars + s);
        bulk_load(dst + ROWS * N1, p.B + row0 * N1, (uint32_t)vec_bytes, bars + s);
    };
    if (tid == 0)
        for (int64_t k = 0; k < NST - 1 && k < mine; ++k) issue_load(k);

    const float gdt = p.lt.gdt;
    const float sixth = 1.0f / 6.0f, third = 1.0f / 3.0f, half = 0.5f;
    const bool vtime = p.lt.pot == PM_TABLE && p.lt.V_nt > 1;
    const PairedTwiddles tw{tw_hi, tw_lo};
    const SwizzledLine L{};
    // a line's exchanges involve only its own T threads: one warp, or a named
    // barrier per line (ids 1..ROWS), so the lines of an item drift apart and
    // one line's arithmetic overlaps another's exchanges
    using LineSync = std::conditional_t<(T <= 32), SyncWarp, SyncNamed>;
    LineSync sync{};
    if constexpr (T > 32) sync = SyncNamed{1 + line, T};

    for (int64_t k = 0; k < mine; ++k) {
        const int s = (int)(k % NST);
        // every thread waits for the stage; the CTA gives up together if any timed out
        const bool landed = mbar_wait(bars + s, (uint32_t)((k / NST) & 1), kWaitNs);
        if (!__syncthreads_and(landed)) {
            uint32_t par[NST];
            for (int q = 0; q < NST; ++q) par[q] = (uint32_t)(((k + (q - s + NST) % NST) / NST) & 1);
            give_up(p.status, bars, par);
            return;
        }
        const int64_t row0 = (blockIdx.x + k * gridDim.x) * ROWS;
        const int64_t row = row0 + line;
        const int64_t path = row / p.n0;
        const int i0 = (int)(row - path * p.n0);
        const uint32_t gp = (uint32_t)(p.lt.path_offset + path);
        V *lineA = bufs + (size_t)s * 2 * ROWS * N1 + line * N1;
        V *lineB = lineA + ROWS * N1;
        V *const sm2[2] = {lineA, lineB};

        // 3D lattices: line i0 of a path is the point pair (i0 / nmid, i0 % nmid)
        const int la = p.ndim == 3 ? i0 / p.nmid : i0;
        const int lb = p.ndim == 3 ? i0 - la * p.nmid : 0;
        // the potential of potential() written out per dimension (no indexed
        // coordinate array, which a run-time dimension count would put in
        // local memory)
        auto pot = [&](int m, uint64_t gs) -> float {
            const int i1 = t + m * T;
            if (p.lt.pot == PM_HARMONIC) {
                const float xa = p.lt.xmin[0] + (float)la * p.lt.dx[0];
                const float xb = p.lt.xmin[1] + (float)(p.ndim == 3 ? lb : i1) * p.lt.dx[1];
                float v = 0.0f;
                v += p.lt.hw2[0] * xa * xa;
                v += p.lt.hw2[1] * xb * xb;
                if (p.ndim == 3) {
                    const float xc = p.lt.xmin[2] + (float)i1 * p.lt.dx[2];
                    v += p.lt.hw2[2] * xc * xc;
                }
                return v;
            }
            if (p.lt.pot == PM_TABLE) {
                int64_t r = p.lt.V_nt > 1 ? (int64_t)gs : 0;
                if (r >= p.lt.V_nt) r = p.lt.V_nt - 1;
                return p.lt.V[r * p.lt.npts + (int64_t)i0 * N1 + i1];
            }
            return 0.0f;
        };
        float Vst[E];
#pragma unroll
        for (int m = 0; m < E; ++m) Vst[m] = vtime ? 0.0f : pot(m, 0);
        auto potv = [&](int m, uint64_t gs) -> float { return vtime ? pot(m, gs) : Vst[m]; };
        auto pterm = [&](int m, uint64_t gs) -> PointTerm<float> {
            if constexpr (NOISE) {
                return point_term(p.lt, potv(m, gs), (uint32_t)(i0 * N1 + t + m * T), gp, (uint32_t)gs);
            } else {
                PointTerm<float> pt;
                pt.dtV = p.lt.dt * potv(m, gs);
                pt.na = make_float2(0.0f, 0.0f);
                return pt;
            }
        };

        V x[2][E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            x[0][m] = lineA[t + m * T];
            x[1][m] = lineB[t + m * T];
        }
        sync();   // the line's natural-order reads complete before swizzled exchanges
        fftp_bwd<N1, E, 2>(x, t, sm2, L, sync, tw);
        if constexpr (MODE == ROW_STAGE2) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const PointTerm<float> pt = pterm(m, p.sg);
                const V aI = x[0][m], k1 = x[1][m];
                const V k2 = apply_N(caxpy(aI, half, k1), pt, gdt);
                const V k3 = apply_N(caxpy(aI, half, k2), pt, gdt);
                x[0][m] = cadd(aI, k3);
                x[1][m] = caxpy(caxpy(caxpy(aI, sixth, k1), third, k2), third, k3);
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) x[0][m] = caxpy(x[1][m], sixth, apply_N(x[0][m], pterm(m, p.sg), gdt));
            if constexpr (SAMPLE) {
                double acc[2] = {0.0, 0.0};
#pragma unroll
                for (int m = 0; m < E; ++m) {
                    const double m2 = (double)cabs2(x[0][m]);
                    acc[0] += m2;
                    acc[1] += (double)potv(m, p.sg + 1) * m2 + 0.5 * p.sm.g * m2 * m2;
                    if ((p.sm.which & (MOM_MOD2 | MOM_MOD4)) && p.sm.per_point &&
                        XSDE_IN((int64_t)p.sample_slot * p.lt.npts + (int64_t)i0 * N1 + t + m * T,
                                p.sm.nsamp * p.lt.npts, p.status)) {
                        double *pp = p.sm.per_point + 2 * ((int64_t)p.sample_slot * p.lt.npts + (int64_t)i0 * N1 + t + m * T);
                        atomicAdd(pp, m2 * p.sm.inv_paths);
                        atomicAdd(pp + 1, m2 * m2 * p.sm.inv_paths);
                    }
                }
                line_sum2<T>(acc, t, line, scratch);
                if (t == 0) {
                    if ((p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path &&
                        XSDE_IN((int64_t)p.sample_slot * p.npaths + path, p.sm.nsamp * p.npaths, p.status)) {
                        double *pq = p.sm.per_path + 2 * ((int64_t)p.sample_slot * p.npaths + path);
                        atomicAdd(pq, acc[0] * p.sm.dV);
                        atomicAdd(pq + 1, acc[1] * p.sm.dV);
                    }
                    if (!isfinite(acc[0])) atomicOr(p.status, ST_NONFINITE);
                }
            }
#pragma unroll
            for (int m = 0; m < E; ++m) x[1][m] = apply_N(x[0][m], pterm(m, p.sg + 1), gdt);
        }
        fftp_fwd<N1, E, 2>(x, t, sm2, L, sync, tw);
        // the dimension-1 factor of exp(L dt/2) (hi/lo: a factor whose FP32
        // rounding misses its modulus by ~6e-8 would scale the populated modes
        // by that at every step); results back in natural order
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + m * T;
            const V eh = e1_s[j], el = e1_s[N1 + j];
            lineA[j] = cmul_hilo(x[0][m], eh, el);
            lineB[j] = cmul_hilo(x[1][m], eh, el);
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            V *src = bufs + (size_t)s * 2 * ROWS * N1;
            if (XSDE_IN(row0 + ROWS - 1, p.npaths * (int64_t)p.n0, p.status)) {
                bulk_store(p.A + row0 * N1, src, (uint32_t)vec_bytes);
                bulk_store(p.B + row0 * N1, src + ROWS * N1, (uint32_t)vec_bytes);
            }
            bulk_commit();
            if (k + NST - 1 < mine) {
                bulk_wait_read<1>();     // the stage of item k-1 has been read out
                issue_load(k + NST - 1);
            }
        }
    }
    if (tid == 0) bulk_wait<0>();
}

// ---------------------------------------------------------------------------
// Column pass
// ---------------------------------------------------------------------------
template <int N0> struct ColTma {
    static constexpr int C = COL_TMA_C;                   // 64-byte row segments
    static constexpr int E = N0 >= 512 ? 16 : 8;
    static constexpr int T = N0 / E;                      // threads per column
    // independent CTAs per SM overlap their phases: 16 warps per SM
    static constexpr int CTAS_PER_SM = 512 / (C * T);
    static constexpr int THREADS = C * T;
    static constexpr int BOXR = N0 < 256 ? N0 : 256;      // tensor-copy box rows
    static constexpr size_t ITEM = (size_t)N0 * C * sizeof(V);
    static constexpr size_t SMEM = NST * ITEM + (size_t)N0 * sizeof(TW) + (size_t)2 * N0 * sizeof(V) +
                                   (THREADS / 32 + 1) * sizeof(double) + NST * sizeof(uint64_t);
};

// TRIG: dimension 0 is a cosine / sine dimension (XMDS2 Sec. 2.1): rows are
// taken from the tile in the even-odd order of the DCT-II's evaluation by an
// N0-point FFT (slot s <- row 2s below N0/2, row 2 N0-1-2s above; odd rows
// negated for the sine basis) and one exchange pairs k with N0-k for
// U_k = A_k V_k + B_k V_{N0-k} (A in E0, B in p.B0, read through L1)
template <int N0, bool TRIG = false>
__global__ void __launch_bounds__(ColTma<N0>::THREADS, ColTma<N0>::CTAS_PER_SM)
    col_pass_tma_kernel(const Params2D<float> p, const __grid_constant__ CUtensorMap mapA,
                        const __grid_constant__ CUtensorMap mapB) {
    using Cfg = ColTma<N0>;
    constexpr int C = Cfg::C, E = Cfg::E, T = Cfg::T, BOXR = Cfg::BOXR;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    V *bufs = reinterpret_cast<V *>(smem_raw);
    TW *tw_s = reinterpret_cast<TW *>(smem_raw + NST * Cfg::ITEM);
    V *e0_s = reinterpret_cast<V *>(tw_s + N0);
    double *scratch = reinterpret_cast<double *>(e0_s + 2 * N0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(scratch + Cfg::THREADS / 32 + 1);

    const int tid = threadIdx.x;
    const int c = tid % C, t = tid / C;
    const int tiles = p.n1 / C;
    // two fields (A, B) per tile, or A alone for the semi-implicit scheme
    const int nvec = p.single_field ? 1 : 2;
    const int64_t nitems = p.npaths * (int64_t)tiles * nvec;
    const int64_t mine = nitems > blockIdx.x ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    for (int i = tid; i < N0; i += blockDim.x) {
        tw_s[i] = p.tw0[i];
        e0_s[i] = p.E0[i];
        e0_s[N0 + i] = p.E0[N0 + i];
    }
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(bars + s, 1);
        fence_barrier_init();
    }
    __syncthreads();
    // the tables above are constants; the fields are the previous pass's output
    grid_launch_dependents();
    grid_dependency_wait();

    // item -> (vector, path, column tile)
    auto decode = [&](int64_t k, int &vec, int64_t &path, int &tile) {
        const int64_t it = blockIdx.x + k * gridDim.x;
        vec = nvec == 2 ? (int)(it & 1) : 0;
        const int64_t rest = nvec == 2 ? it >> 1 : it;
        path = rest / tiles;
        tile = (int)(rest - path * tiles);
    };
    auto issue_load = [&](int64_t k) {
        int vec, tile;
        int64_t path;
        decode(k, vec, path, tile);
        const int s = (int)(k % NST);
        V *dst = bufs + (size_t)s * N0 * C;
        const CUtensorMap *map = vec ? &mapB : &mapA;
        // (bounds-checking build: a tile past the field is skipped, the stage
        // completes without bytes)
        if (!XSDE_IN(tile * C + C - 1, p.n1, p.status) || !XSDE_IN(path, p.npaths, p.status)) {
            mbar_arrive(bars + s);
            return;
        }
        mbar_arrive_expect_tx(bars + s, (uint32_t)Cfg::ITEM);
#pragma unroll
        for (int b = 0; b < N0 / BOXR; ++b)
            tma_load_2d(dst + (size_t)b * BOXR * C, map, tile * C, (int)(path * N0 + b * BOXR), bars + s);
    };
    if (tid == 0)
        for (int64_t k = 0; k < NST - 1 && k < mine; ++k) issue_load(k);

    const TwiddleTable<TW> tw{tw_s};
    const ColumnTile<C> L{c};
    const SyncBlock sync{};
    const bool sample = p.sample_slot >= 0;

    for (int64_t k = 0; k < mine; ++k) {
        const int s = (int)(k % NST);
        // every thread waits for the stage; the CTA gives up together if any timed out
        const bool landed = mbar_wait(bars + s, (uint32_t)((k / NST) & 1), kWaitNs);
        if (!__syncthreads_and(landed)) {
            uint32_t par[NST];
            for (int q = 0; q < NST; ++q) par[q] = (uint32_t)(((k + (q - s + NST) % NST) / NST) & 1);
            give_up(p.status, bars, par);
            return;
        }
        int vec, tile;
        int64_t path;
        decode(k, vec, path, tile);
        V *tileb = bufs + (size_t)s * N0 * C;
        V *const sm1[1] = {tileb};

        const bool odd_neg = TRIG && p.basis0 == 2;
        auto row_of = [&](int j) -> int { return !TRIG ? j : (j < N0 / 2 ? 2 * j : 2 * N0 - 1 - 2 * j); };
        V x[1][E];
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + m * T;
            x[0][m] = tileb[row_of(j) * C + c];
            if (odd_neg && j >= N0 / 2) x[0][m] = mk<V>(-x[0][m].x, -x[0][m].y);
        }
        __syncthreads();
        fft<N0, E, -1, 1>(x, t, sm1, L, sync, tw);
        V xq[E];   // partners V_{N0-k} (TRIG)
        if constexpr (TRIG) {
#pragma unroll
            for (int m = 0; m < E; ++m) tileb[L(t + m * T)] = x[0][m];
            __syncthreads();
#pragma unroll
            for (int m = 0; m < E; ++m) xq[m] = tileb[L((N0 - t - m * T) & (N0 - 1))];
            __syncthreads();
        }
        if (sample && vec == 0) {
            // kinetic energy of a_n: sum_k Re(i L(k)) |F psi|^2 dV/(n0 n1); the
            // dimension-1 factor of exp(L dt/2) already applied is divided out
            const int col = tile * C + c;
            const int k1i = col < p.n1 / 2 ? col : col - p.n1;
            const double k1 = p.sm.kscale[1] * k1i;
            const double w = 1.0 / (double)cabs2(p.E1[col]);
            double sacc = 0.0;
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kj = t + m * T;
                if constexpr (TRIG) {
                    // cosine spectrum from the pair, Parseval weight 2 but at k = 0;
                    // sine mode N0-1-k sits at k
                    // (in the field's precision: the sum is accumulated in FP64)
                    float sn, cs;
                    sincospif(-(float)kj / (2.0f * N0), &sn, &cs);
                    const float xr = 0.5f * (cs * (x[0][m].x + xq[m].x) - sn * (x[0][m].y - xq[m].y));
                    const float xi = 0.5f * (cs * (x[0][m].y + xq[m].y) + sn * (x[0][m].x - xq[m].x));
                    const double k0 = p.sm.kscale[0] * (p.basis0 == 1 ? kj : N0 - kj);
                    sacc += (kj == 0 ? 1.0 : 2.0) * (p.sm.h0 + p.sm.h2 * (k0 * k0 + k1 * k1)) *
                            (double)(xr * xr + xi * xi);
                } else {
                    const double k0 = p.sm.kscale[0] * (kj < N0 / 2 ? kj : kj - N0);
                    sacc += (p.sm.h0 + p.sm.h2 * (k0 * k0 + k1 * k1)) * (double)cabs2(x[0][m]);
                }
            }
            sacc = warp_sum(sacc * w);
            if ((tid & 31) == 0) scratch[tid >> 5] = sacc;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int q = 0; q < Cfg::THREADS / 32; ++q) tot += scratch[q];
                if ((p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path &&
                    XSDE_IN((int64_t)p.sample_slot * p.npaths + path, p.sm.nsamp * p.npaths, p.status))
                    atomicAdd(p.sm.per_path + 2 * ((int64_t)p.sample_slot * p.npaths + path) + 1,
                              tot * p.sm.dV / ((double)N0 * p.n1));
            }
            __syncthreads();
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + m * T;
            if constexpr (TRIG)
                x[0][m] = cadd(cmul_hilo(x[0][m], e0_s[j], e0_s[N0 + j]),
                               cmul_hilo(xq[m], __ldg(p.B0 + j), __ldg(p.B0 + N0 + j)));
            else
                x[0][m] = cmul_hilo(x[0][m], e0_s[j], e0_s[N0 + j]);
        }
        fft<N0, E, +1, 1>(x, t, sm1, L, sync, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + m * T;
            tileb[row_of(j) * C + c] = (odd_neg && j >= N0 / 2) ? mk<V>(-x[0][m].x, -x[0][m].y) : x[0][m];
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            const CUtensorMap *map = vec ? &mapB : &mapA;
            if (XSDE_IN(tile * C + C - 1, p.n1, p.status) && XSDE_IN(path, p.npaths, p.status))
#pragma unroll
                for (int b = 0; b < N0 / BOXR; ++b)
                    tma_store_2d(map, tile * C, (int)(path * N0 + b * BOXR), tileb + (size_t)b * BOXR * C);
            bulk_commit();
            if (k + NST - 1 < mine) {
                bulk_wait_read<1>();
                issue_load(k + NST - 1);
            }
        }
    }
    if (tid == 0) bulk_wait<0>();
}

// Launch with programmatic stream serialization: the kernel may start while
// the previous kernel of the stream drains; it waits for that kernel's results
// in grid_dependency_wait() after loading its tables.
template <typename K, typename... Args>
cudaError_t launch_dependent(K kern, int grid, int threads, size_t smem, cudaStream_t s, const Args &...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int N1, int MODE, bool SAMPLE, bool NOISE>
cudaError_t row_tma_launch(const Params2D<float> &p, int grid, cudaStream_t s) {
    using Cfg = RowTma<N1>;
    auto kern = row_pass_tma_kernel<N1, MODE, SAMPLE, NOISE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t items = p.npaths * (int64_t)p.n0 / Cfg::ROWS;
    const int g = (int)(items < grid ? items : grid);
    return launch_dependent(kern, g, Cfg::THREADS, Cfg::SMEM, s, p);
}

template <int N0>
cudaError_t col_tma_launch(const Params2D<float> &p, const CUtensorMap &a, const CUtensorMap &b, int grid,
                           cudaStream_t s) {
    using Cfg = ColTma<N0>;
    auto kern = p.basis0 ? col_pass_tma_kernel<N0, true> : col_pass_tma_kernel<N0, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t items = p.npaths * (int64_t)(p.n1 / Cfg::C) * (p.single_field ? 1 : 2);
    const int64_t want = (int64_t)grid * Cfg::CTAS_PER_SM;
    const int g = (int)(items < want ? items : want);
    return launch_dependent(kern, g, Cfg::THREADS, Cfg::SMEM, s, p, a, b);
}

}  // namespace

bool tma_row_supported(int n1) { return n1 == 128 || n1 == 256 || n1 == 512 || n1 == 1024; }
bool tma_col_supported(int n0) { return n0 == 128 || n0 == 256 || n0 == 512; }

template <int N1> cudaError_t row_tma_dispatch(int mode, const Params2D<float> &p, int grid, cudaStream_t s) {
    const bool noise = p.lt.noise != NM_NONE, sample = p.sample_slot >= 0;
    if (mode == ROW_STAGE2)
        return noise ? row_tma_launch<N1, ROW_STAGE2, false, true>(p, grid, s)
                     : row_tma_launch<N1, ROW_STAGE2, false, false>(p, grid, s);
    if (sample)
        return noise ? row_tma_launch<N1, ROW_STEADY, true, true>(p, grid, s)
                     : row_tma_launch<N1, ROW_STEADY, true, false>(p, grid, s);
    return noise ? row_tma_launch<N1, ROW_STEADY, false, true>(p, grid, s)
                 : row_tma_launch<N1, ROW_STEADY, false, false>(p, grid, s);
}

cudaError_t launch_row_pass_tma(int mode, const Params2D<float> &p, int grid, cudaStream_t s) {
    if (mode != ROW_STAGE2 && mode != ROW_STEADY) return cudaErrorInvalidValue;
    switch (p.n1) {
        case 128: return row_tma_dispatch<128>(mode, p, grid, s);
        case 256: return row_tma_dispatch<256>(mode, p, grid, s);
        case 512: return row_tma_dispatch<512>(mode, p, grid, s);
        case 1024: return row_tma_dispatch<1024>(mode, p, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_pass_tma(const Params2D<float> &p, const CUtensorMap &a, const CUtensorMap &b, int grid,
                                cudaStream_t s) {
    switch (p.n0) {
        case 128: return col_tma_launch<128>(p, a, b, grid, s);
        case 256: return col_tma_launch<256>(p, a, b, grid, s);
        case 512: return col_tma_launch<512>(p, a, b, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

size_t col_tma_box_rows(int n0) { return n0 < 256 ? (size_t)n0 : 256; }

}  // namespace xsde
