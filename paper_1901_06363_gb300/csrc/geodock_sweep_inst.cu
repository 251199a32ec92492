// Sweep-kernel instantiations for one angle-chunk size GD_KC (candidate
// angles a lane keeps in registers). The build compiles this file once per
// size (GD_KC = 8, 12, 18, 36) into separate objects, so the instantiations
// compile in parallel; each object defines launch_sweep_kc<GD_KC> and
// occupancy_kc<GD_KC>. The exact score (mode 2) is instantiated at 12 only.
#include "geodock_launch.h"

#ifndef GD_KC
#error "compile with -DGD_KC=<angles per chunk>"
#endif

#define GD_CAT2(a, b) a##b
#define GD_CAT(a, b) GD_CAT2(a, b)

namespace gd {

namespace {

template <int MODE, bool CLIP>
cudaError_t go(const SweepParams& P, int grid, int block, size_t smem, cudaStream_t s) {
    auto fn = sweep_kernel<GD_KC, MODE, CLIP>;
    fn<<<grid, block, smem, s>>>(P);
    return cudaGetLastError();
}

template <int MODE, bool CLIP>
cudaError_t occ(int block, size_t smem, int* n) {
    // allow the largest opt-in shared memory once, so every plan's launch fits
    auto fn = sweep_kernel<GD_KC, MODE, CLIP>;
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

constexpr bool kExact = GD_KC == 12;  // the only chunk size with the exact score

}  // namespace

cudaError_t GD_CAT(launch_sweep_kc, GD_KC)(const SweepParams& P, int mode, int clip, int grid, int block, size_t smem,
                                           cudaStream_t s) {
    if (mode == 0) return clip ? go<0, true>(P, grid, block, smem, s) : go<0, false>(P, grid, block, smem, s);
    if (mode == 1) return clip ? go<1, true>(P, grid, block, smem, s) : go<1, false>(P, grid, block, smem, s);
#if GD_KC == 12
    if (mode == 2) return clip ? go<2, true>(P, grid, block, smem, s) : go<2, false>(P, grid, block, smem, s);
#endif
    return cudaErrorInvalidValue;
}

cudaError_t GD_CAT(occupancy_kc, GD_KC)(int mode, int clip, int block, size_t smem, int* n) {
    if (mode == 0) return clip ? occ<0, true>(block, smem, n) : occ<0, false>(block, smem, n);
    if (mode == 1) return clip ? occ<1, true>(block, smem, n) : occ<1, false>(block, smem, n);
#if GD_KC == 12
    if (mode == 2) return clip ? occ<2, true>(block, smem, n) : occ<2, false>(block, smem, n);
#endif
    return cudaErrorInvalidValue;
}

}  // namespace gd
