// Launch description of the body-level smooth-union forward (ccm_union.cu).
#pragma once
#include "../../include/ccm.h"
#include "ccm_device.cuh"

namespace ccm {

struct UnionLaunch {
  DevGeom g;
  const PairRec* pairs;
  const int32_t* row_pair;   // [G] pair << 1 | side of every output group
  int64_t G;
  const float* pose_a;
  const float* pose_b;
  KParams kp;
  float* y;                  // [G, 8]
  int n_sm;
};

cudaError_t launch_union_forward(const UnionLaunch& L, cudaStream_t stream);

}  // namespace ccm
