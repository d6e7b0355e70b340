// Launch description of the per-contact reverse kernels (ccm_flat.cu).
#pragma once
#include "../../include/ccm.h"
#include "ccm_device.cuh"
#include "ccm_clist.cuh"

namespace ccm {

// Scratch of one reverse pass (T = float or Dual) over a contact list of
// capacity cap and G output groups; sizes from flat_pass_bytes.
struct FlatPass {
  void* cval;      // [cap, 8] T: per contact f, d_c, p (3), grad phi (3), SDF frame
  void* force;     // [cap, 6] T: per contact its force and torque on the pair (world)
  void* coef;      // [G] Coef<T>: per group the adjoint coefficients
  void* oterm;     // [G, 6] T: per group the output-transform terms (w, v) of its SDF body
  int* sched;      // [3] work counters of the two per-contact kernels and the fallback
                   // flag (1: the list overflowed or belongs to another forward),
                   // all three set by the pass's first kernel
};

struct FlatLaunch {
  DevGeom g;
  const PairRec* pairs;
  const int32_t* row_pair;   // [G] pair << 1 | side of every output group
  int64_t n_pairs;
  int64_t G;
  const float* pose_a;
  const float* pose_b;
  const float* ybar;         // [G, 8]
  const float* dir;          // [n, 12] or NULL (T = float)
  const float* saved;        // [G, kSavedFloats] record of the forward
  KParams kp;
  ContactList cl;
  FlatPass fp;
  float* grad;               // [n, 12]
  float* hvp;                // [n, 12] or NULL
  float* jvp;                // [G, 8] or NULL
  unsigned long long* counters;   // optional work counters (CCM_BWD_CNT_*)
  int n_sm;
  int pdl;                   // launch the stages with programmatic dependent launch
  int* fallback_sched = nullptr;   // optional: the per-pair kernel's work counter, zeroed
                                   // by the gate kernel (that kernel runs behind the pass)
};

// Bytes of one pass's scratch (FlatPass) for capacity cap and G groups.
void flat_pass_bytes(bool dual, int64_t cap, int64_t G, size_t* cval, size_t* force,
                     size_t* coef, size_t* oterm);
// Tiles of the scan of G group counts (ContactList::tile_sum holds 2 per tile).
int64_t flat_scan_tiles(int64_t G);
// The scan alone: offsets from the group counts (which it zeroes, leaving
// them as cursors), the totals and the tag.
cudaError_t launch_flat_prep_scan(const ContactList& cl, int64_t G, cudaStream_t stream,
                                  bool pdl = false);
// After a forward that filled cl: scan of the group counts and the scatter
// of the records into their fixed order.
cudaError_t launch_flat_prep(const ContactList& cl, int64_t G, int n_sm, cudaStream_t stream);
// The reverse pass from the sorted list (T = Dual when L.dir is set); every
// kernel returns at once when the list overflowed.
cudaError_t launch_flat_backward(const FlatLaunch& L, cudaStream_t stream);

}  // namespace ccm
