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
  Serving* serving = nullptr;

  DevGeom dev_geom() const;
  ccm_status body_of(ccm_geom h, int32_t* idx) const;
  void shutdown_serving();
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
  DevBuf d_pairs;                // pair table
  DevBuf d_order;                // units by decreasing estimated cost
  DevBuf d_part;                 // [2n, 24] per-unit slots of the reverse pass
  BatchMaxima mx;
  ccm_tuning tuning{};
  UnitShape us{};
  int grid = 1;
  int bwd_grid_f = 1, bwd_grid_d = 1;
  void release();
};

ccm_status fail(ccm_status s, const char* fmt, ...);
ccm_status cuda_fail(cudaError_t e, const char* what);
ccm_status make_kparams(const ccm_params* p, KParams* k);
ccm_status build_batch(Context* c, int64_t n, const ccm_geom* A, const ccm_geom* B, Batch* bt);
void default_tuning(ccm_tuning* t);
ccm_status apply_tuning(Context* c, Batch* bt, const ccm_tuning& t);
ccm_status run_forward(Batch* b, const float* pose_a, const float* pose_b, const ccm_params* prm,
                       float* y, unsigned long long* counters, cudaStream_t stream);
ccm_status run_backward(Batch* b, const float* pose_a, const float* pose_b, const ccm_params* prm,
                        const float* ybar, const float* dir, float* grad, float* hvp, float* jvp,
                        cudaStream_t stream);

}  // namespace ccm
