// Sweep-kernel instantiations with 12 candidate angles per register chunk.
#include "geodock_launch.h"

namespace gd {

template <int MODE, bool CLIP>
static cudaError_t go(const SweepParams& P, int grid, int block, size_t smem, cudaStream_t s) {
    auto fn = sweep_kernel<12, MODE, CLIP>;
    fn<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_sweep_kc12(const SweepParams& P, int mode, int clip, int grid, int block, size_t smem,
                               cudaStream_t s) {
    if (mode == 0) return clip ? go<0, true>(P, grid, block, smem, s) : go<0, false>(P, grid, block, smem, s);
    if (mode == 2) return clip ? go<2, true>(P, grid, block, smem, s) : go<2, false>(P, grid, block, smem, s);
    return clip ? go<1, true>(P, grid, block, smem, s) : go<1, false>(P, grid, block, smem, s);
}

template <int MODE, bool CLIP>
static cudaError_t occ(int block, size_t smem, int* n) {
    // allow the largest opt-in shared memory once, so every plan's launch fits
    auto fn = sweep_kernel<12, MODE, CLIP>;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    if (smem > (size_t)optin) {
        *n = 0;
        return cudaSuccess;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, fn, block, smem);
}

cudaError_t occupancy_kc12(int mode, int clip, int block, size_t smem, int* n) {
    if (mode == 0) return clip ? occ<0, true>(block, smem, n) : occ<0, false>(block, smem, n);
    if (mode == 2) return clip ? occ<2, true>(block, smem, n) : occ<2, false>(block, smem, n);
    return clip ? occ<1, true>(block, smem, n) : occ<1, false>(block, smem, n);
}

}  // namespace gd
