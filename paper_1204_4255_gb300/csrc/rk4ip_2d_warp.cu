// rk4ip_2d_warp.cu -- the complex64 column pass with warp-synchronous transforms.
//
// Same arithmetic as rk4ip_2d.cu (XMDS2 Sec. 2.6: exp(L dt/2) applied in
// Fourier space between real-space RK4 stages; Sec. 2.2: the transform of a
// tensor-product lattice factorises per dimension), organised so that no
// transform waits on another warp:
//   column pass : 8-column tiles of A or B (64-byte rows, 64-byte TMA swizzle)
//                 stream through a ring of shared-memory stages; each warp owns
//                 two (or four) columns of the tile and transforms them with the
//                 two-stage plan of fft2.cuh, exchanging in place inside its own
//                 columns.  The last warp to finish a tile stores it and refills
//                 the stage; several small CTAs per SM keep the SM busy while one
//                 of them waits.
//
// Every wait is bounded by the global timer; a wait that runs out records
// ST_TIMEOUT, lets the CTA's other warps stop, waits (bounded) for this CTA's
// copies in flight and returns.
#include <type_traits>

#include "fft2.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace xsde {
namespace {

using V = float2;
using TW = float4;
constexpr uint64_t kWaitNs = 2000000000ull;   // give up on a copy after 2 s

// Wait for phase `parity` of `bar`; false once `abort_flag` is set or the
// time limit passes.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, const volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (global_timer_ns() - t0 > kWaitNs) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Column pass
// ---------------------------------------------------------------------------
template <int N0> struct ColW {
    static constexpr int E = N0 >= 256 ? N0 / 16 : 16;        // points per lane: 32 / 16 / 16
    static constexpr int P = N0 / E;                           // lanes per column: 16 / 16 / 8
    static constexpr int C = WARP_COL_C;                       // tile columns (64-byte rows)
    static constexpr int CPW = 32 / P;                         // columns per warp
    static constexpr int NW = C / CPW;                         // warps per CTA: 4 / 4 / 2
    static constexpr int THREADS = NW * 32;
    static constexpr int NST = N0 == 512 ? 2 : 3;              // shared-memory stages (3 at 512: no faster)
    static constexpr int BOXR = N0 < 256 ? N0 : 256;           // tensor-copy box rows
    static constexpr size_t TILE = (size_t)N0 * C * sizeof(V); // 32 / 16 / 8 KB
    static constexpr int NTW = warp_fft_table_size<N0, E>();
    // (512 points: a compact (c, s) copy of the twiddles for the forward, NTW float2)
    static constexpr size_t TWF = N0 > 256 ? NTW * sizeof(float2) : 0;
    static constexpr size_t SMEM = 1024 + NST * TILE + NTW * sizeof(TW) + 2 * N0 * sizeof(V) + TWF +
                                   NST * (sizeof(uint64_t) + sizeof(long long) + sizeof(int)) + 16;
    static constexpr int CTAS_PER_SM = N0 == 512 ? 2 : N0 == 256 ? 3 : 6;
    static_assert(CTAS_PER_SM * (SMEM + 1024) <= 233472, "shared memory per SM");
};

// The stage ring has no producer warp: thread 0 fills the first stages, and
// the last warp to finish a tile (an arrival count per stage) stores it and
// refills its stage with the tile NST items later.  A bulk store's completion
// is tracked per thread, so that warp also waits until its store has read the
// stage before the load reuses it.
template <int N0>
__global__ void __launch_bounds__(ColW<N0>::THREADS, ColW<N0>::CTAS_PER_SM)
    col_pass_warp_kernel(const Params2D<float> p, const __grid_constant__ CUtensorMap mapA,
                         const __grid_constant__ CUtensorMap mapB) {
    using Cfg = ColW<N0>;
    constexpr int E = Cfg::E, P = Cfg::P, C = Cfg::C, CPW = Cfg::CPW, NW = Cfg::NW, NST = Cfg::NST,
                  BOXR = Cfg::BOXR;
    extern __shared__ unsigned char smem_raw[];
    // tiles start on a 1024-byte boundary (the swizzle pattern repeats every 512)
    unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char *tiles = base;
    TW *tw_s = reinterpret_cast<TW *>(base + NST * Cfg::TILE);
    V *e0_s = reinterpret_cast<V *>(tw_s + Cfg::NTW);
    float2 *twf_s = reinterpret_cast<float2 *>(e0_s + 2 * N0);          // e0_s: hi[N0] | lo[N0]
    uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(twf_s) + Cfg::TWF);
    volatile long long *issued = reinterpret_cast<volatile long long *>(full + NST);   // last item loaded per stage
    int *done = reinterpret_cast<int *>(const_cast<long long *>(issued) + NST);         // warps finished per stage
    volatile int *abort_flag = done + NST;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_per_path = p.n1 / C;
    // two fields (A, B) per tile, or A alone for the semi-implicit scheme
    const int nvec = p.single_field ? 1 : 2;
    const int64_t nitems = p.npaths * (int64_t)tiles_per_path * nvec;
    const int64_t mine = nitems > blockIdx.x ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    // columns of 128 and 256 points (shared-memory-bound at 16 points a lane)
    // stage the paired twiddles as split (c, s) / (c eps, s eps) arrays, so the
    // forward reads 8 bytes a lane at an 8-byte stride; 512 keeps float4 entries
    // for the backward (one 16-byte read a twiddle) and a compact (c, s) copy
    // for the forward
    constexpr bool SPLIT = N0 <= 256;
    float2 *tw_hi = reinterpret_cast<float2 *>(tw_s), *tw_lo = tw_hi + Cfg::NTW;
    if constexpr (SPLIT) {
        stage_paired(tw_hi, tw_lo, p.tw0w, Cfg::NTW, tid, blockDim.x);
    } else {
        for (int i = tid; i < Cfg::NTW; i += blockDim.x) {
            const TW w = p.tw0w[i];
            tw_s[i] = w;
            twf_s[i] = make_float2(w.x, w.y);
        }
    }
    for (int i = tid; i < 2 * N0; i += blockDim.x) e0_s[i] = p.E0[i];
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(full + s, 1);
            issued[s] = -1;
            done[s] = 0;
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    // the tables above are constants; the fields are the previous pass's output
    grid_launch_dependents();
    grid_dependency_wait();

    // item -> (vector, path, column tile)
    auto decode = [&](int64_t k, int &vec, int64_t &path, int &tile) {
        const uint32_t it = (uint32_t)(blockIdx.x + k * gridDim.x);
        vec = nvec == 2 ? (int)(it & 1) : 0;
        const uint32_t rest = nvec == 2 ? it >> 1 : it;
        const uint32_t pth = rest / (uint32_t)tiles_per_path;
        path = pth;
        tile = (int)(rest - pth * (uint32_t)tiles_per_path);
    };
    auto issue_load = [&](int64_t k) {
        int vec, tile;
        int64_t path;
        decode(k, vec, path, tile);
        const int s = (int)(k % NST);
        unsigned char *dst = tiles + (size_t)s * Cfg::TILE;
        issued[s] = k;
        // (bounds-checking build: a tile past the field is skipped, the stage
        // completes without bytes)
        if (!XSDE_IN(tile * C + C - 1, p.n1, p.status) || !XSDE_IN(path, p.npaths, p.status)) {
            mbar_arrive(full + s);
            return;
        }
        mbar_arrive_expect_tx(full + s, (uint32_t)Cfg::TILE);
#pragma unroll
        for (int b = 0; b < N0 / BOXR; ++b)
            tma_load_2d(dst + (size_t)b * BOXR * (C * 8), vec ? &mapB : &mapA, tile * C, (int)(path * N0 + b * BOXR),
                        full + s);
    };
    auto issue_store = [&](int64_t k) {
        int vec, tile;
        int64_t path;
        decode(k, vec, path, tile);
        const unsigned char *src = tiles + (size_t)(k % NST) * Cfg::TILE;
        if (XSDE_IN(tile * C + C - 1, p.n1, p.status) && XSDE_IN(path, p.npaths, p.status))
#pragma unroll
            for (int b = 0; b < N0 / BOXR; ++b)
                tma_store_2d(vec ? &mapB : &mapA, tile * C, (int)(path * N0 + b * BOXR),
                             src + (size_t)b * BOXR * (C * 8));
        bulk_commit();
    };
    // leave on a copy that never lands: record it, stop the CTA's other warps
    // and wait (bounded) for the loads in flight and this thread's stores
    auto give_up = [&]() {
        if (lane == 0) {
            atomicOr(p.status, ST_TIMEOUT);
            *abort_flag = 1;
            for (int s = 0; s < NST; ++s) {
                const long long kk = issued[s];
                if (kk >= 0) mbar_wait(full + s, (uint32_t)((kk / NST) & 1), kWaitNs);
            }
            bulk_wait<0>();
        }
        __syncwarp();
    };
    if (tid == 0)
        for (int64_t k = 0; k < NST && k < mine; ++k) issue_load(k);

    // The warp owns columns warp * CPW .. + CPW-1.  Eight-byte shared accesses
    // are served in two 16-lane phases, so each phase must span all of the
    // warp's columns (a column's rows reach only 8 of the 16 bank pairs of a
    // swizzled 128-byte row): two columns alternate lane by lane; four columns
    // take lanes in blocks of 8 (each half-warp then holds two columns).
    const int c = CPW == 2 ? warp * 2 + (lane & 1) : warp * CPW + lane / P;
    const int t = CPW == 2 ? lane >> 1 : lane % P;
    const auto tw = [&] {
        if constexpr (SPLIT) return PairedTwiddles{tw_hi, tw_lo};
        else return TwiddleTable<TW>{tw_s};
    }();
    // the forward's twiddles: the (c, s) halves only (tw_fwd reads no more)
    const auto twf = [&] {
        if constexpr (SPLIT) return PairedTwiddles{tw_hi, tw_lo};
        else return PairedTwiddles{twf_s, twf_s};
    }();
    const bool sample = p.sample_slot >= 0;
    for (int64_t k = 0; k < mine; ++k) {
        const int s = (int)(k % NST);
        if (!wait_or_abort(full + s, (uint32_t)((k / NST) & 1), abort_flag)) {
            give_up();
            return;
        }
        int vec, tile;
        int64_t path;
        decode(k, vec, path, tile);
        unsigned char *tb = tiles + (size_t)s * Cfg::TILE;
        // element (row, c) of the tile as the 64-byte swizzle lays it out: in
        // 64-byte rows, 16-byte chunk (c / 2) ^ ((row / 2) % 4)
        auto at = [&](int row) -> V * {
            return reinterpret_cast<V *>(tb + 64 * row + ((((c >> 1) ^ ((row >> 1) & 3))) << 4) + ((c & 1) << 3));
        };
        auto xat = [&](int i) -> V * { return at(xslot<E>(i)); };
        V x[E];
#pragma unroll
        for (int m = 0; m < E; ++m) x[m] = *at(t + P * m);
        __syncwarp();
        warp_fft<N0, E>(x, t, xat, twf);
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
                const int kj = t + P * m;
                const double k0 = p.sm.kscale[0] * (kj < N0 / 2 ? kj : kj - N0);
                sacc += (p.sm.h0 + p.sm.h2 * (k0 * k0 + k1 * k1)) * (double)cabs2(x[m]);
            }
            sacc = warp_sum(sacc * w);
            if (lane == 0 && (p.sm.which & (MOM_NORM | MOM_ENERGY)) && p.sm.per_path &&
                XSDE_IN((int64_t)p.sample_slot * p.npaths + path, p.sm.nsamp * p.npaths, p.status))
                atomicAdd(p.sm.per_path + 2 * ((int64_t)p.sample_slot * p.npaths + path) + 1,
                          sacc * p.sm.dV / ((double)N0 * p.n1));
        }
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + P * m;
            x[m] = cmul_hilo(x[m], e0_s[j], e0_s[N0 + j]);
        }
        warp_ifft<N0, E>(x, t, xat, tw);
#pragma unroll
        for (int m = 0; m < E; ++m) *at(t + P * m) = x[m];
        // the tile goes out through the tensor-memory-access unit (async proxy)
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(done + s, 1) == NW - 1) {
                // every warp has written its columns of the tile
                atomicExch(done + s, 0);
                __threadfence_block();
                issue_store(k);
                if (k + NST < mine) {
                    bulk_wait_read<0>();
                    issue_load(k + NST);
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0) bulk_wait<0>();
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

template <int N0>
cudaError_t col_warp_launch(const Params2D<float> &p, const CUtensorMap &a, const CUtensorMap &b, int num_sms,
                            cudaStream_t s) {
    using Cfg = ColW<N0>;
    auto kern = col_pass_warp_kernel<N0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    const int64_t items = p.npaths * (int64_t)(p.n1 / Cfg::C) * (p.single_field ? 1 : 2);
    const int64_t want = (int64_t)num_sms * Cfg::CTAS_PER_SM;
    const int g = (int)(items < want ? items : want);
    return launch_dependent(kern, g, Cfg::THREADS, Cfg::SMEM, s, p, a, b);
}

}  // namespace

bool warp_col_supported(int n0, int64_t n1) { return (n0 == 128 || n0 == 256 || n0 == 512) && n1 % WARP_COL_C == 0; }
int warp_col_elems(int n0) { return n0 >= 256 ? n0 / 16 : 16; }
size_t warp_col_box_rows(int n0) { return n0 < 256 ? (size_t)n0 : 256; }

cudaError_t launch_col_pass_warp(const Params2D<float> &p, const CUtensorMap &a, const CUtensorMap &b, int num_sms,
                                 cudaStream_t s) {
    if (!p.tw0w || p.basis0) return cudaErrorInvalidValue;
    switch (p.n0) {
        case 128: return col_warp_launch<128>(p, a, b, num_sms, s);
        case 256: return col_warp_launch<256>(p, a, b, num_sms, s);
        case 512: return col_warp_launch<512>(p, a, b, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace xsde
