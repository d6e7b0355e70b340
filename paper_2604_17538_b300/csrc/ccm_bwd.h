// Launch description of the reverse-pass kernels (ccm_bwd.cu).
//
// Adjoint of one contact c of a group with blend weight w_c = f_c om_c,
// om_c = exp(-d_c / tau_blend) / sum_j f_j exp(-d_j / tau_blend), where the
// group's outputs are d = sum w d_c, a = sum w f_c, q = sum w p_c and
// nu = sum w grad phi_c (S frame; the world point is R_S q + t_S and the
// normal R_S nu / |nu|):
//   g_c   = dbar d_c + abar f_c + qbar . p_c + nubar . grad phi_c,
//   gbar  = dbar d + abar a + qbar . q + nubar . nu,
//   fbar  = w abar + (g_c - gbar) om_c,
//   dcbar = w (dbar - (g_c - gbar) / tau_blend),
//   phibar = dcbar (f + f' (phi - d_max)) + fbar f',
//   xbar  = w qbar + phibar grad phi + w H nubar,
// with qbar = R_S^T pbar_w and nubar = (nbar_S - n_S (n_S . nbar_S)) / |nu|.
#pragma once
#include "../../include/ccm.h"
#include "ccm_device.cuh"
#include "ccm_unit.cuh"

namespace ccm {

struct BwdLaunch {
  DevGeom g;
  const PairRec* pairs;
  const WorkItem* items;      // work items (unit, feature-piece range)
  const int32_t* order;       // item indices by decreasing estimated cost
  int64_t n_items;
  const int64_t* item_off;    // [n_pairs + 1] items of pair p: [item_off[p], item_off[p+1])
  int64_t n_pairs;
  const int64_t* dev_items;   // if set: entries of `order` to run, read on device
  const int64_t* dev_pairs;   // if set: pairs to reduce, read on device
  const float* pose_a;
  const float* pose_b;
  const float* ybar;    // [G, 8]
  const float* dir;     // [n, 12] or NULL
  const float* saved;   // [G, kSavedFloats] from the forward with these poses, or NULL
  const int32_t* pair_order;   // pairs by decreasing cost: with `saved`, run per pair
                               // (every SDF body <= kHitS pieces), else NULL
  KParams kp;
  UnitShape us;
  float* part;          // [n_items, 24] per-item slots (workspace)
  float* grad;          // [n, 12]
  float* hvp;           // [n, 12] or NULL
  float* jvp;           // [G, 8] or NULL
  unsigned long long* counters;   // optional work counters (CCM_BWD_CNT_*)
  int* sched;                     // optional work counter (device int), zeroed by the launch
  int grid;        // one-warp blocks of the per-item kernel
  int pair_grid;   // one-warp blocks of the per-pair kernel
  // if set: the per-pair kernel runs only when this device word is non-zero
  // (the per-contact kernels did not run: see FlatPass::sched)
  const int* only_if = nullptr;
  // behind the per-contact pass: the per-pair kernel is launched with
  // programmatic dependent launch (it waits for the pass before it reads
  // only_if), and `sched` was zeroed by the pass (no memset)
  bool after_chain = false;
};

// Resident one-warp blocks per SM of the reverse kernels that launch_backward
// uses for a shape, indexed [T: 0 float, 1 Dual][trace steps: 0 any, 1 three].
struct BwdOccupancy {
  int unit[2][2];
  int pair[2][2];
};

cudaError_t launch_backward(const BwdLaunch& L, cudaStream_t stream);
cudaError_t configure_backward(const UnitShape& us, int smem_limit, BwdOccupancy* occ);
int backward_slice_bytes(const UnitShape& us, bool dual);

// Variant with the per-item slots in a fixed device array (no workspace).
cudaError_t launch_backward_noalloc(BwdLaunch L, int device, cudaStream_t stream);
int64_t noalloc_max_items();

}  // namespace ccm
