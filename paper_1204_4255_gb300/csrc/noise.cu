// noise.cu -- the Wiener-noise generator exposed on its own: raw Philox4x32-10
// words and the Box-Muller normal pairs a step draws (XMDS2 Sec. 2.5; Philox
// after Salmon et al., SC'11).  The integrators call the same device functions.
#include "kernels.h"

namespace xsde {
namespace {

__global__ void philox_kernel(const uint4 *ctr, uint2 key, int64_t n, uint4 *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], key);
}

template <typename R>
__global__ void normals_kernel(uint2 key, int64_t npts, int64_t npaths, int64_t path_offset, uint32_t step,
                               cx<R> *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts * npaths) return;
    const int64_t p = i / npts, j = i - p * npts;
    out[i] = wiener_pair<R>(key, (uint32_t)j, (uint32_t)(path_offset + p), step);
}

}  // namespace

cudaError_t launch_philox(const uint32_t *ctr, uint64_t seed, int64_t n, uint32_t *out, cudaStream_t s) {
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const int64_t blocks = (n + 255) / 256;
    if (blocks > 0)
        philox_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const uint4 *>(ctr), key, n,
                                                       reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_normals(uint64_t seed, int64_t npts, int64_t npaths, int64_t path_offset, uint32_t step,
                           void *out, cudaStream_t s) {
    const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const int64_t blocks = (npts * npaths + 255) / 256;
    if (blocks > 0)
        normals_kernel<R><<<(unsigned)blocks, 256, 0, s>>>(key, npts, npaths, path_offset, step,
                                                          static_cast<cx<R> *>(out));
    return cudaGetLastError();
}

template cudaError_t launch_normals<float>(uint64_t, int64_t, int64_t, int64_t, uint32_t, void *, cudaStream_t);
template cudaError_t launch_normals<double>(uint64_t, int64_t, int64_t, int64_t, uint32_t, void *, cudaStream_t);

}  // namespace xsde
