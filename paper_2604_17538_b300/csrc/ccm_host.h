// Host-side objects behind the opaque handles of include/ccm.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ccm.h"
#include "ccm_device.cuh"
#include "ccm_fwd.h"
#include "ccm_bwd.h"
#include "ccm_flat.h"
#include "ccm_union.h"
#include "ccm_spline.h"
#include "ccm_ffwd.h"

namespace ccm {

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  void release();
};

struct Serving;   // continuous-batching request loop (ccm_serve.cu)

struct Context {
  int device = 0;
  size_t budget = 0;
  int n_sm = 0;
  int smem_optin = 0;
  std::mutex mu;
  // host mirror of the resident geometry (append-only; handles stay stable)
  std::vector<PieceRec> pieces;
  std::vector<BodyRec> bodies;
  std::vector<float4> verts;
  std::vector<float4> planes;
  std::vector<uint32_t> edges;
  std::vector<uint8_t> alive;
  DevBuf d_pieces, d_bodies, d_verts, d_planes, d_edges;
  // tricubic spline SDFs (ccm_attach_splines): one record per piece (zero
  // dims when it has none) and the coefficient rows
  std::vector<SplineRec> splines;
  std::vector<float4> spline_coef;
  DevBuf d_splines, d_spline_coef;
  // broad-phase voxel grids (ccm_build_voxel_grids): one record per piece
  // loaded when they were built
  DevBuf d_voxels, d_voxel_vals;
  int64_t n_voxels = 0;
  Serving* serving = nullptr;

  DevGeom dev_geom() const;
  ccm_status body_of(ccm_geom h, int32_t* idx) const;
  void shutdown_serving();
};

// Device buffers, side streams and events of ccm_contacts_step_host.
struct HostStep {
  DevBuf pa, pb, y, saved, ybar, grad, grad2, hvp, dir, jvp;
  cudaStream_t cin = nullptr, cout = nullptr;   // input and output copies
  cudaEvent_t ev[5] = {};   // pose copy / end, inputs, forward, H u pass, gradient pass
  void release();
};

struct BatchMaxima {      // largest pieces / bodies a batch touches
  int vmax = 1, fmax = 1, emax = 1, s_planes = 1, s_pieces = 1, f_verts = 1, f_edges = 1;
  int pieces_any = 1;
};

struct Batch {
  Context* ctx = nullptr;
  int64_t n = 0;
  int64_t G = 0;
  std::vector<int64_t> goff;
  std::vector<PairRec> pairs;    // host copy of the pair table
  DevBuf d_pairs;                // pair table
  int64_t n_items = 0;
  DevBuf d_items;                // work items (depend on the tuning)
  DevBuf d_item_order;           // item indices by decreasing estimated cost
  DevBuf d_item_off;             // [n + 1] items of each pair
  DevBuf d_part;                 // [n_items, 24] per-item slots of the reverse pass
  DevBuf d_pair_order;           // pairs by decreasing cost (per-pair reverse pass)
  bool per_pair = false;         // every body has <= kHitS pieces
  DevBuf d_sched;                // [3] work counters: forward, gradient pass, H u pass
  DevBuf d_status;               // [1] CCM_ERR_TIMEOUT once a bounded wait ran out
  BatchMaxima mx;
  ccm_tuning tuning{};
  UnitShape us{};
  int grid = 1;
  BwdOccupancy bwd_occ{};        // reverse kernels' resident blocks per SM
  HostStep* hs = nullptr;        // ccm_contacts_step_host state (first call)
  // contact list of ccm_contacts_save and the per-contact reverse passes
  // (ccm_flat.cu); flat_cap = 0: none
  int64_t flat_cap = 0;
  uint32_t list_tag = 0;         // tag of the last contact list (0: none yet)
  DevBuf d_row_pair;             // [G] pair << 1 | side
  DevBuf d_fctl, d_fcnt, d_foff, d_frecs, d_fsorted, d_ftiles;
  DevBuf d_fpass[2][5];          // [float, Dual][cval, force, coef, oterm, sched]
  // flat forward (ccm_ffwd.cu): directions per unit, relative poses, live
  // directions, candidate contacts and their values, the list's values
  int64_t n_dirs = 0, cand_cap = 0;
  DevBuf d_unit_dir_off, d_rel, d_live, d_cand, d_cand_m, d_cval, d_sval, d_skey, d_ffctl,
      d_ffhits;
  ContactList contact_list() const;
  FlatPass flat_pass(bool dual) const;
  void release();
};

ccm_status fail(ccm_status s, const char* fmt, ...);
ccm_status cuda_fail(cudaError_t e, const char* what);

#define CCM_CUDA(call, what)                           \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)
ccm_status make_kparams(const ccm_params* p, KParams* k);
BatchMaxima body_maxima(const Context& c, int32_t body);
void merge_maxima(BatchMaxima* m, const BatchMaxima& b);
// A run of feature pieces [fc0, fc1) of one body that one work item covers
// (at most us.groups pieces within the vertex and edge budgets), with its
// vertex + edge count.
struct PieceChunk {
  uint16_t fc0, fc1;
  int64_t feats;
};
void body_chunks(const Context& c, int32_t body, const UnitShape& us,
                 std::vector<PieceChunk>* out);
// The items (and estimated costs) of unit `unit` from its feature body's
// chunks against an SDF body of s_np pieces.
void push_items(const std::vector<PieceChunk>& chunks, int32_t unit, int32_t s_np,
                std::vector<WorkItem>* items, std::vector<int64_t>* cost);
// Work items of the n pairs for shape `us`, appended in pair order: unit
// indices are 2 (unit_pair0 + i) + side; cost[] gets each item's estimated
// cost and item_off[] (if not NULL) the running item count after each pair.
void make_items(const Context& c, const PairRec* pairs, int64_t n, int64_t unit_pair0,
                const UnitShape& us, std::vector<WorkItem>* items, std::vector<int64_t>* cost,
                std::vector<int64_t>* item_off);
// Item indices by decreasing cost (ties: index order).
std::vector<int32_t> items_by_cost(const std::vector<int64_t>& cost);
ccm_status build_batch(Context* c, int64_t n, const ccm_geom* A, const ccm_geom* B, Batch* bt);
void default_tuning(ccm_tuning* t);
ccm_status apply_tuning(Context* c, Batch* bt, const ccm_tuning& t);
// (Re)allocates the contact list and the per-contact passes' scratch for the
// batch's tuning (flat_records), or releases them.
ccm_status setup_flat(Context* c, Batch* bt);
ccm_status run_forward(Batch* b, const float* pose_a, const float* pose_b, const ccm_params* prm,
                       float* y, float* saved, unsigned long long* counters, cudaStream_t stream);
ccm_status run_backward(Batch* b, const float* pose_a, const float* pose_b, const ccm_params* prm,
                        const float* saved, const float* ybar, const float* dir, float* grad,
                        float* hvp, float* jvp, unsigned long long* counters,
                        cudaStream_t stream);

}  // namespace ccm
