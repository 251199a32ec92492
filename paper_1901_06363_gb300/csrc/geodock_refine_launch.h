// Host launchers of the refinement and differentiable-score kernels.
#pragma once

#include <cuda_runtime.h>

#include "geodock_refine.cuh"

namespace gd {

enum ScoreLaunch { SCORE_FWD = 0, SCORE_BWD = 1, DOF_APPLY = 2, DOF_GRAD = 3 };

// One warp per (pocket, ligand) pair; lmax / tmax: largest atom / torsion count of the batch.
cudaError_t launch_refine(const RefineParams& P, int lmax, int tmax, cudaStream_t s);

// One warp per ligand: trilinear o (SCORE_FWD), its adjoint (SCORE_BWD), the
// pose update z(q) (DOF_APPLY) or its adjoint J(q)^T dL/dz (DOF_GRAD).
cudaError_t launch_score(const ScoreParams& P, int lmax, int which, cudaStream_t s);

}  // namespace gd
