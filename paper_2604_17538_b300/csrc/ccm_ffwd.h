// Launch description of the flat forward (ccm_ffwd.cu).
#pragma once
#include "../../include/ccm.h"
#include "ccm_device.cuh"
#include "ccm_clist.cuh"
#include "ccm_flat.h"

namespace ccm {

// control words: live directions, vertex and edge candidates (vertices fill
// the first half of the candidate arrays, edges the second, so that a warp of
// the eval stage takes contacts of one kind), overflow flag
enum { kFfLive = 0, kFfCand = 1, kFfOverflow = 2, kFfSched = 3, kFfCandE = 4, kFfWords = 8 };

// largest piece (in planes) for which the gate stages the SDF body's planes
// in shared memory; a batch with larger pieces gates from global memory
constexpr int kGateStageMaxPlanes = 256;

struct FlatFwdLaunch {
  DevGeom g;
  const PairRec* pairs;
  const int32_t* row_pair;        // [G] pair << 1 | side
  const int64_t* unit_dir_off;    // [2n + 1] directions of the units before unit u
  int64_t n_pairs, G, n_dirs;
  const float* pose_a;
  const float* pose_b;
  KParams kp;
  float* y;                       // [G, 8]
  float* saved;                   // [G, kSavedFloats] or NULL
  uint32_t* hits;                 // [G, kHitWords] hit words while the forward runs
  ContactList cl;                 // the contact list it fills (sorted, counts, offsets)
  float* sval;                    // [cl.cap, 8] contact values, in list order
  long long* sval_key;            // [cl.cap] (SDF piece, feature) keys, in arrival order
  float* rel;                     // [2n, 12] relative poses S <- F per unit
  int4* live;                     // [n_dirs] live directions (row, F piece, S piece, plane)
  int64_t cand_cap;
  int4* cand;                     // [cand_cap] candidate contacts (row, S piece, F piece, w)
  float2* cand_m;                 // [cand_cap] max-plane lower bounds (vertex; edge corners)
  float* cval;                    // [cand_cap, 8] contact values
  unsigned long long* ctl;        // [kFfWords]
  unsigned long long* counters;   // optional CCM_CNT_* work counters
  int vmax;                       // most vertices of a feature piece in the batch
  int fmax;                       // most planes of a piece in the batch
  int gate_planes;                // planes staged per gate warp (>= fmax), or 0: the gate
                                  // reads the planes from global memory
  int stage_tma;                  // stage planes with bulk copies on an mbarrier (1) or loads
  long long wait_limit;           // polls of a bulk copy's barrier before giving up
  int* status;                    // CCM_ERR_TIMEOUT when a wait gave up
  int pdl;                        // launch the stages with programmatic dependent launch
  int n_sm;
  int* fallback_sched = nullptr;  // optional: the per-item kernel's work counter, zeroed
                                  // by the setup stage (that kernel runs behind the chain)
};

// Runs the flat forward.  When its candidate or contact list overflows, its
// last kernels do nothing and ctl[kFfOverflow] is set: the caller then runs
// the per-item forward kernel (gated on that word).
cudaError_t launch_flat_forward(const FlatFwdLaunch& L, cudaStream_t stream);
size_t flat_forward_feature_smem(int vmax, int fmax, int* warps_per_block);
// whether a batch's largest pieces fit the flat forward's shared-memory staging
bool flat_forward_fits(int vmax, int fmax);

}  // namespace ccm
