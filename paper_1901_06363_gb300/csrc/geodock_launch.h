// Launchers of the sweep-kernel instantiations (one translation unit per
// angle-chunk size so they compile in parallel).
#pragma once
#include <cuda_runtime.h>

#include "geodock_kernels.cuh"

namespace gd {

// Returns the CUDA error of the launch (or of the attribute/occupancy query).
cudaError_t launch_sweep_kc8(const SweepParams& P, int mode, int clip, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_sweep_kc12(const SweepParams& P, int mode, int clip, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_sweep_kc18(const SweepParams& P, int mode, int clip, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t launch_sweep_kc36(const SweepParams& P, int mode, int clip, int grid, int block, size_t smem, cudaStream_t s);

}  // namespace gd

namespace gd {
cudaError_t occupancy_kc8(int mode, int clip, int block, size_t smem, int* n);
cudaError_t occupancy_kc12(int mode, int clip, int block, size_t smem, int* n);
cudaError_t occupancy_kc18(int mode, int clip, int block, size_t smem, int* n);
cudaError_t occupancy_kc36(int mode, int clip, int block, size_t smem, int* n);
}  // namespace gd
