// Launch description of the tricubic spline-SDF forward (ccm_spline.cu).
#pragma once
#include "../../include/ccm.h"
#include "ccm_device.cuh"

namespace ccm {

struct SplineLaunch {
  DevGeom g;
  const SplineRec* splines;  // [pieces] of the context
  const float4* coef;        // coefficient rows of the context
  const PairRec* pairs;
  const int32_t* row_pair;   // [G] pair << 1 | side of every output group
  int64_t G;
  const float* pose_a;
  const float* pose_b;
  KParams kp;
  float* y;                  // [G, 8]
  int n_sm;
};

cudaError_t launch_spline_forward(const SplineLaunch& L, cudaStream_t stream);

}  // namespace ccm
