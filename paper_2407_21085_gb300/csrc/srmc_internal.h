// srmc_internal.h -- declarations shared by the translation units of libsrmc.
#pragma once

#include "srmc_device.cuh"

namespace srmc {

// Model variants of the step kernel: the driver needs z only for the cos
// model with kapz != 0 and for the logistic model.
enum ModelVariant { MV_COS = 0, MV_COS_Z = 1, MV_LOGISTIC = 2, MV_AFFINE = 3 };

#define SRMC_LAUNCH_STEP_NAME(D) SRMC_LAUNCH_STEP_NAME_(D)
#define SRMC_LAUNCH_STEP_NAME_(D) launch_step_d##D

#define SRMC_DECLARE_STEP(D)                                                              \
    cudaError_t launch_step_d##D(const Params &P, int i, bool fp64, bool lp1, int mv, int grid, \
                                 int threads, cudaStream_t st);
SRMC_DECLARE_STEP(1)
SRMC_DECLARE_STEP(2)
SRMC_DECLARE_STEP(3)
SRMC_DECLARE_STEP(4)
SRMC_DECLARE_STEP(5)
SRMC_DECLARE_STEP(6)
SRMC_DECLARE_STEP(7)
SRMC_DECLARE_STEP(8)
#undef SRMC_DECLARE_STEP

}  // namespace srmc
