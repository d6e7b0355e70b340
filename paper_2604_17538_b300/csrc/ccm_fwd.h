// Launch description of the forward kernels (ccm_fwd.cu).
#pragma once
#include "../../include/ccm.h"
#include "ccm_device.cuh"
#include "ccm_unit.cuh"
#include "ccm_clist.cuh"

namespace ccm {

struct FwdLaunch {
  DevGeom g;
  const PairRec* pairs;
  const WorkItem* items;  // work items (unit, feature-piece range)
  const int32_t* order;   // item indices by decreasing estimated cost
  int64_t n_items;
  const int64_t* dev_items;   // if set: number of entries of `order` to run, read on device
  const float* pose_a;
  const float* pose_b;
  KParams kp;
  UnitShape us;
  float* y;
  float* saved;                   // optional [G, kSavedFloats] for the reverse pass
  unsigned long long* counters;   // optional work counters (CCM_CNT_*)
  int* sched;                     // optional work counter (device int), zeroed by the launch
  int grid;
  ContactList cl{};               // with `saved`: the contact list (cl.recs NULL: none)
  int* status = nullptr;          // optional device word: CCM_ERR_TIMEOUT if a bounded wait ran out
  // if set: the kernel runs only when this device word is non-zero (the flat
  // forward overflowed)
  const unsigned long long* only_if = nullptr;
  // behind the flat forward's chain: launched with programmatic dependent
  // launch (the kernel waits for the chain before it reads only_if), and
  // `sched` was zeroed by the chain (no memset)
  bool after_chain = false;
};

cudaError_t launch_forward(const FwdLaunch& L, cudaStream_t stream);
cudaError_t configure_forward(const UnitShape& us, int smem_limit, int* blocks_per_sm);

}  // namespace ccm
