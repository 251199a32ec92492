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

namespace gd {
// Measured rates (geodock_peaks.cu): r[0] scalar FP32 FMA/s, r[1] packed
// FP32 FMA/s (two per instruction), r[2] texture fetches/s over the whole
// field, r[3] texture fetches/s within 16^3-voxel cubes, r[4] random 32-byte
// L2 sector loads/s. tex: the padded field's texture, px x py x pz voxels.
cudaError_t measure_peaks(unsigned long long tex, int px, int py, int pz, int num_sms, cudaStream_t s, double* r);
}  // namespace gd
