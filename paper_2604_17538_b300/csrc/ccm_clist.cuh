// The contact list a forward keeps for the per-contact reverse kernels
// (ccm_flat.cu): every contact of non-zero weight (Sec. 4.3: f_t > 0), one
// record each, so that the reverse passes revisit exactly the contacts that
// enter a blend (Sec. 4.4) instead of re-gating and re-culling every piece
// pair.  Records hold indices only; the SDF is recomputed, never stored.
//
// The forward appends records in no fixed order (one atomic per warp round)
// and counts the contacts of every output group, vertices and edges apart; a
// record carries its rank among its group's contacts of its kind, in the
// order the forward found them.  A scan of the counts and a scatter then put
// the records in a fixed order: every vertex contact (by group, then rank),
// then every edge contact -- so a group's and a pair's contacts are
// contiguous, and every reduction over them runs in an order that depends on
// the pair alone.
//
// The list lives in the batch, the saved record with the caller.  Every
// forward that keeps a list gives it a new tag and writes the tag into the
// saved record too; a reverse pass uses the list only when the record's tag
// matches it (and the list did not overflow), else it falls back to the
// record's hit marks.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccm {

// record word w: bit 31 edge (1) or vertex (0); bits 19..30 the feature's
// piece-local index; bits 0..18 the rank within (group, kind)
constexpr int kRankBits = 19;
constexpr int kFeatBits = 12;

struct ContactList {
  int4* recs;               // [cap] (row, S piece, F piece, w), appended by the forward
  int4* sorted;             // [cap] (row, S piece, F piece, feature | kind << 31), fixed order
  int64_t cap;
  unsigned long long* ctl;  // [8]: appended, overflow flag, vertex contacts NV, edge contacts NE,
                            // the list's tag
  uint32_t tag;             // this forward's tag (non-zero), also kept in every saved row
  int32_t* cnt_v;           // [G] vertex contacts per group
  int32_t* cnt_e;           // [G] edge contacts per group
  int32_t* off_v;           // [G + 1] exclusive prefix of cnt_v
  int32_t* off_e;           // [G + 1] exclusive prefix of cnt_e
  int32_t* live_g;          // [G] the groups with at least one contact, in index order
  long long* tile_sum;      // [2 tiles] scratch of the scan (flat_scan_tiles)
};

// ctl words: appended records, overflow flag, vertex contacts NV, edge
// contacts NE, the list's tag, groups with contacts NG
enum { kCtlCursor = 0, kCtlOverflow = 1, kCtlNV = 2, kCtlNE = 3, kCtlTag = 4, kCtlNG = 5,
       kCtlWords = 8 };

}  // namespace ccm
