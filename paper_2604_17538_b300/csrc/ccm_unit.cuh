// The forward pass of one unit (pair, side) for one warp: the N_F blend groups
// of body F's convex pieces against the pieces of body S (Sec. 4.2-4.4).
//
// Work is flattened so that all 32 lanes stay busy although only a few
// features of a live piece pair survive the exact culls:
//   * S's planes and F's vertices (moved into S's frame) and edges are staged
//     in the warp's shared-memory slice -- in chunks when a body is large;
//   * directions (f, s) are gated 32 at a time (lane per direction) and the
//     live ones are collected in (f, s) order into a pending list;
//   * for a list of live directions, the max-plane pass runs over all their
//     (direction, vertex) items, the edge cull over all (direction, edge)
//     items, and the SDF evaluations over the compacted survivors of all of
//     them; items stay sorted by group, so after each round of 32 contacts a
//     segmented warp reduction (online softmax) folds them into the groups'
//     accumulators kept in shared memory -- one head lane per group, in a
//     fixed order, so the result is deterministic.
#pragma once
#include "ccm_blend.cuh"

namespace ccm {

// Per-batch budgets of the per-warp shared-memory slice.
struct UnitShape {
  int32_t plane_budget;   // planes of one S chunk (>= largest piece)
  int32_t spiece_budget;  // pieces of one S chunk
  int32_t vert_budget;    // vertices of one F chunk (>= largest piece)
  int32_t edge_budget;    // edges of one F chunk (>= largest piece)
  int32_t item_v;         // (direction, vertex) items per direction list
  int32_t item_e;         // (direction, edge) items per direction list
  int32_t slice_bytes;    // bytes per warp
  int32_t warps;          // warps per block
  int32_t groups;         // feature pieces (groups) per chunk, <= kGroupsPerChunk
  int32_t item_vb;        // item budgets of the reverse pass
  int32_t item_eb;
  int32_t groups_b;       // groups per chunk of the reverse pass (<= groups)
  int32_t hit_words;      // hit words per group kept in shared memory:
                          // ceil(largest S body's pieces / 32) <= kHitWords
  int32_t stage_tma;      // 1: stage the SDF body's planes with bulk copies (TMA)
  int64_t wait_limit;     // iterations of a bounded wait for a bulk copy
};

constexpr int kGroupsPerChunk = 32;   // most groups of one F chunk (lane-indexed)
constexpr int kPending = 32;          // live directions per list

struct UnitSlice {
  float4* planes;     // [plane_budget]
  int2* sp;           // [spiece_budget] (first plane, plane count) per S piece
  float4* xs;         // [vert_budget] F vertices in the S frame
  uint32_t* edges;    // [edge_budget]
  int4* fp;           // [groups] (first vertex, nv, first edge, ne) per F piece
  float4* fs;         // [groups] bounding sphere (S frame) per F piece
  PartT<float>* acc;  // [groups] group blend partials (ccm_blend.cuh)
  uint32_t* hit;      // [groups * hw] directions that gave a contact
  int hw;             // hit words per group (UnitShape::hit_words)
  int* dir;           // [32] pending live directions: fc << 16 | sc
  int* dsub;          // [32] directions of the list being run
  int* dpl;           // [32] per pending direction: a plane attaining the gate's max
  int* dsubpl;        // [32] the same for the list being run
  int* pv;            // [33] prefix of vertex items per pending direction
  int* pe;            // [33] prefix of edge items
  float* m;           // [item_v] max-plane value per (direction, vertex)
  float* phi;         // [item_v] SDF per (direction, vertex) (from the vertex contacts on)
  uint16_t* vlist;    // [item_v] surviving vertex items
  uint16_t* elist;    // [item_e] surviving edge items
  uint8_t* need;      // [item_v]
  float* vb;          // [item_v] voxel-grid lower bound of the SDF per (direction, vertex)
  uint16_t* am;       // [item_v] a plane attaining the max-plane value (until the
                      // edge cull, in phi's space)
  int* gcnt;          // [2 groups] contacts of non-zero weight per group (vertex,
                      // edge) found so far, for the contact list
  uint64_t* mbar;     // [1] completion barrier of the warp's bulk copies
};

// Rounding allowance of the edge cull's plane bound (coordinates are O(1) in
// the SDF frame, so float rounding of the bound is ~1e-7).
constexpr float kEdgeTol = 1e-5f;
// Voxel-grid culls: the same allowance, and the flag in a vertex item's
// plane index that says the grid culled it (plane indices are < 1024).
constexpr float kVoxTol = 1e-5f;
constexpr uint16_t kVoxCulled = 0x8000;
constexpr uint16_t kPlaneMask = 0x7fff;

__host__ __device__ inline int align16i(int b) { return (b + 15) & ~15; }

__host__ __device__ inline int unit_slice_bytes(const UnitShape& u) {
  int b = 0;
  b += 16 * u.plane_budget;
  b += align16i(8 * u.spiece_budget);
  b += 16 * u.vert_budget;
  b += align16i(4 * u.edge_budget);
  b += 16 * u.groups;                        // fp
  b += 16 * u.groups;                        // fs
  b += align16i((int)sizeof(PartT<float>) * u.groups);   // acc
  b += align16i(4 * u.hit_words * u.groups);   // hit
  b += align16i(4 * kPending) * 4;           // dir, dsub, dpl, dsubpl
  b += align16i(4 * (kPending + 1)) * 2;     // pv, pe
  b += align16i(4 * u.item_v) * 2;           // m, phi
  b += align16i(2 * u.item_v);               // vlist
  b += align16i(2 * u.item_e);               // elist
  b += align16i(u.item_v);                   // need
  b += align16i(4 * u.item_v);               // vb
  b += align16i(8 * u.groups);               // gcnt
  b += 16;                                   // mbar
  return b;
}

__device__ inline UnitSlice unit_slice(unsigned char* p, const UnitShape& u) {
  UnitSlice s;
  s.planes = reinterpret_cast<float4*>(p);           p += 16 * u.plane_budget;
  s.sp = reinterpret_cast<int2*>(p);                 p += align16i(8 * u.spiece_budget);
  s.xs = reinterpret_cast<float4*>(p);               p += 16 * u.vert_budget;
  s.edges = reinterpret_cast<uint32_t*>(p);          p += align16i(4 * u.edge_budget);
  s.fp = reinterpret_cast<int4*>(p);                 p += 16 * u.groups;
  s.fs = reinterpret_cast<float4*>(p);               p += 16 * u.groups;
  s.acc = reinterpret_cast<PartT<float>*>(p);        p += align16i((int)sizeof(PartT<float>) * u.groups);
  s.hit = reinterpret_cast<uint32_t*>(p);            p += align16i(4 * u.hit_words * u.groups);
  s.hw = u.hit_words;
  s.dir = reinterpret_cast<int*>(p);                 p += align16i(4 * kPending);
  s.dsub = reinterpret_cast<int*>(p);                p += align16i(4 * kPending);
  s.dpl = reinterpret_cast<int*>(p);                 p += align16i(4 * kPending);
  s.dsubpl = reinterpret_cast<int*>(p);              p += align16i(4 * kPending);
  s.pv = reinterpret_cast<int*>(p);                  p += align16i(4 * (kPending + 1));
  s.pe = reinterpret_cast<int*>(p);                  p += align16i(4 * (kPending + 1));
  s.m = reinterpret_cast<float*>(p);                 p += align16i(4 * u.item_v);
  s.phi = reinterpret_cast<float*>(p);               p += align16i(4 * u.item_v);
  s.vlist = reinterpret_cast<uint16_t*>(p);          p += align16i(2 * u.item_v);
  s.elist = reinterpret_cast<uint16_t*>(p);          p += align16i(2 * u.item_e);
  s.need = reinterpret_cast<uint8_t*>(p);             p += align16i(u.item_v);
  s.vb = reinterpret_cast<float*>(p);                 p += align16i(4 * u.item_v);
  s.gcnt = reinterpret_cast<int*>(p);               p += align16i(8 * u.groups);
  s.mbar = reinterpret_cast<uint64_t*>(p);
  s.am = reinterpret_cast<uint16_t*>(s.phi);
  return s;
}

// largest r in [0, n) with pre[r] <= t (pre is an exclusive prefix, pre[0] = 0)
__device__ __forceinline__ int find_dir(const int* pre, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace ccm
