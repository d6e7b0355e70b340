/*
 * ccm.h -- C ABI of the B300-native contact-manifold library.
 *
 * One-shot smooth contact manifolds between rigid bodies that are decomposed
 * into convex pieces (arxiv 2604.17538, Sec. 4).  For every body pair and every
 * pair of convex pieces the library runs an exact broad-phase cull and the
 * smooth gate of Sec. 4.3, evaluates vertex-SDF and sphere-traced edge-SDF
 * contacts (Sec. 4.2) against each piece's smooth polytope SDF (Sec. 3: LSE
 * over the half-space SDFs of the piece), and blends the contacts of each
 * convex piece into one contact (Sec. 4.4, N_1 + N_2 contacts per body pair).
 *
 * Conventions shared by every entry point
 *   - Status codes only; nothing throws across the ABI.  On failure
 *     ccm_last_error() returns a message for the calling thread.
 *   - Pointers documented as "device" must be device memory of the context's
 *     GPU; "host" pointers are read before the call returns.
 *   - Asynchronous entry points enqueue work on the given stream, never
 *     synchronize and never allocate; an asynchronous CUDA error surfaces as
 *     CCM_ERR_CUDA from a later call.
 *   - Poses are float32 rows of 12: row-major R (9) then t (3), mapping body
 *     frame to world (x_w = R x + t).
 *   - Group outputs are float32 rows of 8: (d, a, p_x, p_y, p_z, n_x, n_y, n_z)
 *     = blended signed depth, blend weight, world contact point, world unit
 *     normal (pointing out of the SDF body).  Pair i owns the groups
 *     [off[i], off[i+1]): first one per piece of body A (A's vertices and
 *     edges against B's pieces), then one per piece of body B.  A group with
 *     no active contact is (d_max, 0, 0, 0, 0, 0, 0, 0).
 *   - Twist coordinates of a pair (derivatives): (w_A, v_A, w_B, v_B), with
 *     R_X <- Exp([w_X]x) R_X, t_X <- t_X + v_X.
 *
 * How the calls map to a per-call signature that passes the pairs each time,
 * ccm_contacts(ctx, n, A[n], B[n], pose_a, pose_b, params, outputs, stream):
 *   - the pair list (A[i], B[i]) is planned once by ccm_batch_create, which
 *     uploads the pair table and the work items and allocates the workspace;
 *     ccm_contacts(batch, pose_a, pose_b, params, y, stream) then takes only
 *     what changes between steps (poses and params), so that it neither
 *     allocates nor synchronises;
 *   - the outputs are one array y[G, 8] (array of structures, the row layout
 *     above) rather than separate depth / weight / point / normal arrays;
 *     the group offsets come from ccm_batch_info (or ccm_output_size);
 *   - the reverse pass takes its cotangents in the same [G, 8] layout and
 *     returns 12 twist components per pair (w_A, v_A, w_B, v_B);
 *   - ccm_poll also returns the request's latency.
 */
#ifndef CCM_H_
#define CCM_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CCM_API __attribute__((visibility("default")))
#else
#define CCM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ccm_ctx_s* ccm_ctx;
typedef struct ccm_batch_s* ccm_batch;
typedef uint64_t ccm_geom;     /* handle of one resident body */
typedef uint64_t ccm_ticket;   /* handle of one submitted request */
typedef void* ccm_stream;      /* a cudaStream_t (0 = legacy default stream) */

typedef enum {
  CCM_OK = 0,
  CCM_ERR_INVALID = 1,        /* bad argument, bad geometry or bad handle */
  CCM_ERR_OOM = 2,            /* device allocation or memory budget exceeded */
  CCM_ERR_CUDA = 3,           /* CUDA runtime error (message has the detail) */
  CCM_ERR_TIMEOUT = 4,        /* a bounded device-side wait ran out */
  CCM_ERR_BUSY = 5,           /* request not admitted now; retry later */
  CCM_ERR_NOT_READY = 6,      /* request still in flight */
  CCM_ERR_UNKNOWN_TICKET = 7  /* ticket never issued or already retired */
} ccm_status;

/* Flags of ccm_params.flags */
#define CCM_FLAG_NO_CULL 1u   /* evaluate every feature (culls are exact; for tests) */
/* Forward variants (ccm_contacts only; the reverse passes and ccm_contacts_save
 * reject them):
 *   BODY_UNION: the other body's SDF is the smooth union of its pieces' SDFs,
 *     phi_S = -tau_sdf log sum_s exp(-phi_s / tau_sdf) (Sec. 3.1, Eq.
 *     soft_union), and every vertex and edge of a group's piece gives one
 *     contact against the whole body instead of one per piece;
 *   PROJECT: every contact point is moved onto the SDF's isosurface,
 *     p - phi(p) grad phi(p) (Sec. 4.1), after its depth and normal were
 *     taken at p. */
#define CCM_FLAG_BODY_UNION 2u
#define CCM_FLAG_PROJECT 4u
/* SPLINE: every SDF piece is its tricubic spline SDF (Sec. 3.2, attached with
 * ccm_attach_splines), and the contact normal is its normal spline; forward
 * only, like the two above, and not combined with BODY_UNION. */
#define CCM_FLAG_SPLINE 8u
/* VOXEL_CULL: the forward also culls with the voxel grids of
 * ccm_build_voxel_grids (Sec. 4.3 broad phase: a vertex whose voxel's lower
 * bound b of the SDF is >= d_max, an edge whose corners' bounds give
 * (b_I + b_II - length) / 2 >= d_max); culls are exact, so outputs equal
 * those without the flag to float rounding.  Without grids the flag changes
 * nothing. */
#define CCM_FLAG_VOXEL_CULL 16u

/* Method constants.  The paper fixes none of these values (Sec. 2-4). */
typedef struct {
  float tau_sdf;      /* LSE softness of the piece SDF (Sec. 3, Eq. smooth-intersection) */
  float tau_trace;    /* softness of the sphere-trace gate [[phi > 0]] (Sec. 4.2) */
  float tau_clip;     /* softness of the edge soft clip (Sec. 2, 4.2) */
  float tau_blend;    /* softmax temperature of the contact blend (Sec. 4.4) */
  float d_max;        /* distance threshold of the broad phase (Sec. 4.3) */
  float gate_width;   /* transition bandwidth epsilon > 0 (Sec. 4.3) */
  int32_t trace_iters;/* sphere-trace iterations, 0..16 (three in Sec. 4.2) */
  uint32_t flags;     /* CCM_FLAG_* */
} ccm_params;

/* Fills *p with the defaults: all softness 5e-3, d_max = 0.01, epsilon = 0.01,
 * 3 trace iterations, no flags. */
CCM_API void ccm_default_params(ccm_params* p);

/* Host description of one body: n_pieces convex pieces, each with nv[i]
 * vertices (xyz), nf[i] face planes (n_x, n_y, n_z, h; n unit outward, so
 * n.x + h < 0 inside, Sec. 3 half-space SDF) and ne[i] edges (pairs of
 * piece-local vertex indices).  Arrays are concatenated over the pieces. */
typedef struct {
  int32_t n_pieces;
  const int32_t* nv;
  const int32_t* nf;
  const int32_t* ne;
  const float* verts;      /* [sum nv, 3] */
  const float* planes;     /* [sum nf, 4] */
  const int32_t* edges;    /* [sum ne, 2] */
} ccm_body_desc;

/* Creates a context on CUDA device `device`.  `hbm_budget_bytes` bounds the
 * device memory the serving loop may admit (0 = no bound).  Errors:
 * CCM_ERR_INVALID (no such device), CCM_ERR_CUDA. */
CCM_API ccm_status ccm_create(int device, size_t hbm_budget_bytes, ccm_ctx* out);

/* Releases every device resource of the context (waits for its work). */
CCM_API void ccm_destroy(ccm_ctx ctx);

/* Message of the last failed call on this thread ("" if none). */
CCM_API const char* ccm_last_error(void);

/* Copies n_bodies bodies into device memory owned by the context and returns
 * one handle per body in out[n_bodies] (host).  Limits: 1..4096 pieces per
 * body, 1..1024 vertices, 4..1024 planes and 0..3072 edges per piece; edge
 * indices must be valid and edges of non-zero length.  Synchronous.
 * Errors: CCM_ERR_INVALID, CCM_ERR_OOM, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_load_geometry(ccm_ctx ctx, const ccm_body_desc* bodies, int n_bodies,
                             ccm_geom* out);

/* Tricubic spline SDFs of one body's convex pieces (Sec. 3.2), for
 * CCM_FLAG_SPLINE.  Piece p has a voxel grid from origin grid[4p..4p+2] with
 * cubic voxels of size grid[4p+3] > 0 and dims[3p..3p+2] voxels per axis
 * (1..256); its spline has (nx+3)(ny+3)(nz+3) coefficient rows of 4 floats
 * (SDF, normal x, y, z), z index fastest, coefficient k of an axis at grid
 * node k - 1, so that s(x) = sum c u(tx - kx + 1) u(ty - ky + 1) u(tz - kz + 1)
 * with t = (x - origin) / h and the paper's basis u.  The pieces' rows are
 * concatenated in `coef`.  Outside its grid box a piece's SDF is the spline
 * at the nearest box point plus the distance to the box.  All host arrays. */
typedef struct {
  const float* grid;       /* [n_pieces, 4] */
  const int32_t* dims;     /* [n_pieces, 3] */
  const float* coef;       /* [sum of rows, 4] */
} ccm_spline_desc;

/* Attaches (or replaces) the spline SDFs of `body`'s pieces, one desc for
 * the whole body.  Synchronous; allocates.  Errors: CCM_ERR_INVALID (bad
 * handle, sizes or non-finite values), CCM_ERR_OOM, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_attach_splines(ccm_ctx ctx, ccm_geom body, const ccm_spline_desc* desc);

/* Builds the broad-phase voxel grids (Sec. 4.3) of every piece loaded so far,
 * for CCM_FLAG_VOXEL_CULL: per piece a grid of cubic voxels over the
 * bounding box of its vertices, `voxels` (1..64) along its longest side,
 * each voxel holding a lower bound of the piece's SDF anywhere in it: the
 * largest plane value at its centre minus its circumradius (the largest
 * plane value is 1-Lipschitz and never above the smooth SDF).  Pieces loaded
 * later have no grid until the next call.  Synchronous; allocates.
 * Errors: CCM_ERR_INVALID, CCM_ERR_OOM, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_build_voxel_grids(ccm_ctx ctx, int voxels);

/* Marks bodies as released: later calls reject their handles.  Batches that
 * were planned before keep working.  Device memory of released bodies is
 * returned when the context is destroyed.  Errors: CCM_ERR_INVALID. */
CCM_API ccm_status ccm_free_geometry(ccm_ctx ctx, const ccm_geom* handles, int n);

/* Number of output groups of the n pairs (A[i], B[i]) (host arrays):
 * sum over pairs of (pieces of A[i] + pieces of B[i]). */
CCM_API ccm_status ccm_output_size(ccm_ctx ctx, int64_t n, const ccm_geom* A, const ccm_geom* B,
                           int64_t* groups);

/* Plans a batch of n body pairs (A[i], B[i]) (host arrays): uploads the pair
 * table and the group offsets and picks the launch shape.  The batch is the
 * unit that ccm_contacts and ccm_contacts_backward run on; poses change
 * between calls, pairs do not.  Calls on one batch share its workspace
 * (reverse-pass slots, work counters): issue them in order on one stream.
 * The one exception: after a ccm_contacts_save, a ccm_contacts_backward_saved
 * without dir and one with dir (separate output buffers) may run
 * concurrently on two streams when every body has at most 256 pieces.
 * Synchronous; allocates.
 * Errors: CCM_ERR_INVALID, CCM_ERR_OOM, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_batch_create(ccm_ctx ctx, int64_t n, const ccm_geom* A, const ccm_geom* B,
                            ccm_batch* out);
CCM_API void ccm_batch_destroy(ccm_batch batch);

/* Number of pairs and of groups of a batch, and (if off != NULL) the group
 * offsets off[n+1] copied to host memory. */
CCM_API ccm_status ccm_batch_info(ccm_batch batch, int64_t* n_pairs, int64_t* n_groups, int64_t* off);

/* Launch shape of a batch.  Each (pair, side) is cut into work items of at
 * most `groups` feature pieces (one warp each, heaviest first), so that large
 * bodies spread over many warps.  The kernels gather the live piece pairs of
 * an item into lists whose vertex and edge items fill the warp's
 * shared-memory budgets below; larger lists keep more lanes busy, smaller ones
 * leave room for more resident warps.  Defaults: 256 / 512 / 256 / 512 items,
 * 2 forward warps per block, 16 groups per work item.  Budgets below the
 * batch's largest piece are raised to it.  Results do not depend on the
 * tuning beyond float rounding order. */
typedef struct {
  int32_t item_v, item_e;     /* forward: vertex / edge items per list */
  int32_t item_vb, item_eb;   /* reverse pass: vertex / edge items per list */
  int32_t fwd_warps;          /* forward warps per block, 1..4 */
  int32_t groups;             /* feature pieces per work item, 1..32 */
  int32_t stage_planes;       /* most SDF-body planes staged at once (0: 1024 per work item,
                                 512 per warp in the flat gate, which takes at most 760;
                                 at least the largest piece's), 0 or 16..4096 */
  int32_t stage_verts;        /* most feature-piece vertices staged at once, edges
                                 3x that (0: 512; at least the largest piece's), 0 or 16..4096 */
  int32_t groups_b;           /* reverse pass: feature pieces per chunk (0: 4; at most
                                 groups), 0..32 */
  int32_t flat_records;       /* capacity of the contact list that ccm_contacts_save keeps
                                 for the per-contact reverse passes, in records per output
                                 group (0: 16, and at least 4,096 in all; -1: no list, the
                                 reverse passes re-gate per pair and the forward runs per
                                 item), -1..4096 */
  int32_t stage_tma;          /* forward (per-item kernel and flat stages): stage the SDF
                                 planes into shared memory with bulk (TMA) copies (0) or
                                 plain loads (-1) */
  int32_t stage_wait;         /* bound of a bulk copy's wait, in polls of its barrier, each
                                 suspending at most 1 us (0: 2^22; -1: none, so that every
                                 wait runs out -- for tests of the timeout path), -1..2^30 */
  int32_t flat_forward;       /* forward as flat stages (gate per direction, culls per live
                                 direction, one contact per thread, fold per group) on a
                                 batch with a contact list (0), or one warp per work item
                                 (-1) */
  int32_t pdl;                /* flat stages launched with programmatic dependent launch,
                                 each stage scheduled while the previous one drains (0), or
                                 as ordinary launches (-1) */
} ccm_tuning;
CCM_API ccm_status ccm_batch_get_tuning(ccm_batch batch, ccm_tuning* out);
/* Synchronous (sets kernel attributes).  Errors: CCM_ERR_INVALID (out of
 * range or too large for shared memory), CCM_ERR_CUDA. */
CCM_API ccm_status ccm_batch_set_tuning(ccm_batch batch, const ccm_tuning* t);

/* Waits for `stream` and reports whether a kernel of the batch stopped on a
 * bounded device-side wait since the last check (CCM_ERR_TIMEOUT; its outputs
 * are then incomplete), clearing the flag.  Synchronous.
 * Errors: CCM_ERR_INVALID, CCM_ERR_TIMEOUT, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_batch_check(ccm_batch batch, ccm_stream stream);

/* Number of kernels the library has launched in this process (every context
 * and stream), counted on the host as they are issued; the kernels of a CUDA
 * graph captured from the library's calls count once, at capture, however
 * often it is replayed.  For measurement.  Errors: CCM_ERR_INVALID (NULL). */
CCM_API ccm_status ccm_kernel_launches(int64_t* n);

/* Forward pass (Sec. 4.2-4.4).  pose_a, pose_b: device [n,12] float32; y:
 * device [G,8] float32, fully overwritten.  Asynchronous on `stream`.
 * Errors: CCM_ERR_INVALID (NULL pointer, bad params), CCM_ERR_CUDA. */
CCM_API ccm_status ccm_contacts(ccm_batch batch, const float* pose_a, const float* pose_b,
                        const ccm_params* prm, float* y, ccm_stream stream);

/* Reverse pass.  Given the cotangent ybar (device [G,8]) of the outputs, writes
 * grad (device [n,12]) = d<ybar, y>/d(twist) at twist = 0.  If dir (device
 * [n,12]) is given, also writes hvp (device [n,12]) = H dir, the Hessian of
 * <ybar, y> in the twist chart applied to dir, and, if jvp != NULL, the output
 * tangents jvp (device [G,8]) = (dy/dtwist) dir.  The per-vertex SDF is
 * recomputed, not stored.  Asynchronous; allocates nothing.
 * Errors: CCM_ERR_INVALID, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_contacts_backward(ccm_batch batch, const float* pose_a, const float* pose_b,
                                 const ccm_params* prm, const float* ybar, const float* dir,
                                 float* grad, float* hvp, float* jvp, ccm_stream stream);

/* Floats per output group of the record ccm_contacts_save keeps for the
 * reverse pass: the group's blend partial, which of the SDF body's pieces
 * gave it a contact of non-zero weight, and the tag of the contact list the
 * same call kept in the batch. */
#define CCM_SAVED_FLOATS 28

/* ccm_contacts that also fills saved (device [G, CCM_SAVED_FLOATS] float32,
 * fully overwritten) for ccm_contacts_backward_saved.  Asynchronous on
 * `stream`.  Errors: CCM_ERR_INVALID, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_contacts_save(ccm_batch batch, const float* pose_a, const float* pose_b,
                                     const ccm_params* prm, float* y, float* saved,
                                     ccm_stream stream);

/* ccm_contacts_backward given the record of a ccm_contacts_save call with the
 * same batch, poses and params: its passes visit only the contacts that had
 * a non-zero weight in the forward pass, the only ones with a non-zero
 * adjoint, instead of re-running the broad phase over all piece pairs.  When
 * every body has at most 256 pieces, ccm_contacts_save also keeps a list of
 * those contacts in the batch (tuning flat_records), and the passes run one
 * contact per thread from it: recompute the contact, blend each group,
 * form its adjoint coefficients, back-propagate each contact into a force
 * and a torque, and sum them per pair in a fixed order.  If the list
 * overflowed (or without it) they revisit, per pair, the (piece, piece)
 * directions the record marks.  Results equal ccm_contacts_backward's up to
 * float rounding order and do not depend on the rest of the batch; a record
 * of other poses (or a list of another ccm_contacts_save of the batch) gives
 * wrong results.  Asynchronous on `stream`.
 * Errors: CCM_ERR_INVALID, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_contacts_backward_saved(ccm_batch batch, const float* pose_a,
                                               const float* pose_b, const ccm_params* prm,
                                               const float* saved, const float* ybar,
                                               const float* dir, float* grad, float* hvp,
                                               float* jvp, ccm_stream stream);

/* One step from host memory, for callers whose poses and cotangents live on
 * the host: copies pose_a, pose_b (host [n,12]) and, if given, ybar (host
 * [G,8]) and dir (host [n,12]) into device buffers the batch owns, runs
 * ccm_contacts_save, then (with ybar) one pass of ccm_contacts_backward_saved:
 * with dir the forward-over-reverse pass, whose gradient (the primal part of
 * its dual numbers) is grad and whose tangents are hvp and jvp, without dir
 * the gradient pass; and copies back y (host
 * [G,8]), grad (host [n,12]; required with ybar) and, with dir, hvp (host
 * [n,12]; required) and jvp (host [G,8]; optional).  Results are those of
 * the device calls on the same data (with dir: grad is that call's grad).
 * The ybar / dir copies run on a second stream during the forward (after the
 * pose copy, which the forward waits for), and y is copied back on a third
 * stream while the reverse pass runs; only the pose copy and the copies of
 * the reverse pass's outputs (or y for a forward alone) are not hidden
 * behind a kernel.  Host
 * buffers should be pinned (cudaHostAlloc, torch pin_memory) so that the
 * copies are asynchronous.  Asynchronous on `stream`: the outputs are
 * complete once the work queued on `stream` up to this call is (synchronize
 * it before reading them); later work on `stream` waits for every copy.  The
 * first call allocates the device buffers (the poses, y, the record, ybar,
 * the gradient, hvp, dir and jvp: 52 n + (8 + CCM_SAVED_FLOATS + 8) G
 * floats) and two streams, kept until ccm_batch_destroy; later calls
 * allocate nothing.  Calls on one batch must be ordered on one stream.
 * Errors: CCM_ERR_INVALID (NULL pointer a mode needs, dir without ybar),
 * CCM_ERR_OOM, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_contacts_step_host(ccm_batch batch, const float* pose_a,
                                          const float* pose_b, const ccm_params* prm,
                                          const float* ybar, const float* dir, float* y,
                                          float* grad, float* hvp, float* jvp,
                                          ccm_stream stream);

/* Same as ccm_contacts_backward, for callers that cannot obtain device
 * memory for scratch -- e.g. code running while another framework owns the
 * whole device memory pool, or a real-time loop that forbids allocation after
 * start-up.  The per-work-item slots of the reverse pass (24 floats each)
 * live in one fixed 4 MiB array compiled into the library instead of the
 * batch's workspace, so the call allocates nothing and uses no workspace;
 * the caller still passes every input and output.  The paper has no
 * counterpart: this is a deployment variant of the same computation.
 *   - Limit: 43690 work items (43690 * 24 floats <= 2^20), i.e. n <= 21845
 *     pairs when no body has more pieces than one work item holds (the
 *     tuning's `groups`); larger batches are rejected with CCM_ERR_INVALID.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *     The address is kept for the life of the process: after a device reset
 *     (cudaDeviceReset, or a framework that destroys and recreates the
 *     device's primary context) it is stale, so do not call this entry point
 *     again in that process.
 *   - Every call on a device shares the array and it keeps the last call's
 *     contents.  Nothing in it needs to start at zero: each call writes every
 *     slot it reads.  Calls that overlap on the GPU (other streams, other
 *     threads) race on it; serialise them.
 * Errors: CCM_ERR_INVALID, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_contacts_backward_noalloc(ccm_batch batch, const float* pose_a,
                                                 const float* pose_b, const ccm_params* prm,
                                                 const float* ybar, const float* dir,
                                                 float* grad, float* hvp, float* jvp,
                                                 ccm_stream stream);

/* Work counters of the last ccm_contacts_counted call, for the roofline:
 * counts of piece-pair directions, surviving directions, plane evaluations by
 * kind and contacts.  Same as ccm_contacts plus device atomics on `counters`
 * (device, CCM_N_COUNTERS int64, zeroed by the caller). */
#define CCM_N_COUNTERS 8
enum {
  CCM_CNT_DIRS = 0,        /* (SDF piece, feature piece) directions examined */
  CCM_CNT_DIRS_LIVE = 1,   /* directions that passed the piece-pair gate */
  CCM_CNT_MAXPASS = 2,     /* plane evaluations of the vertex max pass */
  CCM_CNT_GATEPASS = 3,    /* plane evaluations of the piece-pair gate */
  CCM_CNT_EVAL_GRAD = 4,   /* plane evaluations with exp and gradient */
  CCM_CNT_EVAL_VAL = 5,    /* plane evaluations with exp, value only */
  CCM_CNT_CONTACTS = 6,    /* contacts with a non-zero weight */
  CCM_CNT_FEATURES = 7     /* features examined (vertices + edges) */
};
CCM_API ccm_status ccm_contacts_counted(ccm_batch batch, const float* pose_a, const float* pose_b,
                                const ccm_params* prm, float* y, int64_t* counters,
                                ccm_stream stream);

/* Work counters of one reverse pass, for the roofline: directions examined,
 * directions in lists, and plane evaluations by kind -- pass-1 gate and
 * max-plane tests, pass-1 evaluations with gradient and value-only trace
 * steps, pass-2 evaluations with gradient and Hessian-vector product and
 * pass-2 trace steps with gradient.  Same as ccm_contacts_backward_saved
 * (saved may be NULL: ccm_contacts_backward) plus device atomics on
 * `counters` (device, CCM_N_COUNTERS int64, zeroed by the caller). */
enum {
  CCM_BWD_CNT_DIRS = 0,       /* directions examined by a gate or the hit marks
                                 (per-contact passes: contacts evaluated) */
  CCM_BWD_CNT_DIRS_LIVE = 1,  /* directions run through lists (per-contact passes:
                                 contacts of a group with a non-zero weight) */
  CCM_BWD_CNT_MAXPASS = 2,    /* plane evaluations of the max-plane passes */
  CCM_BWD_CNT_GATEPASS = 3,   /* plane evaluations of piece-pair gates */
  CCM_BWD_CNT_P1_GRAD = 4,    /* pass 1: plane evaluations with gradient */
  CCM_BWD_CNT_P1_VAL = 5,     /* pass 1: value-only trace-step evaluations */
  CCM_BWD_CNT_P2_HV = 6,      /* pass 2: evaluations with gradient and H v */
  CCM_BWD_CNT_P2_GRAD = 7     /* pass 2: trace-step evaluations with gradient */
};
CCM_API ccm_status ccm_contacts_backward_counted(ccm_batch batch, const float* pose_a,
                                                 const float* pose_b, const ccm_params* prm,
                                                 const float* saved, const float* ybar,
                                                 const float* dir, float* grad, float* hvp,
                                                 float* jvp, int64_t* counters, ccm_stream stream);

/* Measures, on `device`, the throughput of the arithmetic units the contact
 * kernels are bound by: FP32 FMA (scalar and packed f32x2, in TFLOP/s, an
 * FMA counted as 2 FLOP) and the SFU's ex2 (in tera-ops/s).  Synchronous;
 * allocates 16 bytes.  Not part of the method: it provides the roofline
 * denominators.  Errors: CCM_ERR_INVALID, CCM_ERR_OOM, CCM_ERR_CUDA. */
CCM_API ccm_status ccm_peak_probe(int device, double* ffma_tflops, double* ffma2_tflops,
                                  double* ex2_tops);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of small requests (Sec. 5 workloads, where
 * many environments each ask for the contacts of a few body pairs).
 *
 * Requests are queued by ccm_submit and packed, first come first served, by a
 * scheduler thread inside the library into waves of at most max_wave_pairs
 * pairs and max_wave_requests requests.  A wave is one replay of a CUDA graph
 * that gathers every request's poses (and cotangents), runs the forward pass
 * over all of the wave's pairs and the reverse pass over the pairs of the
 * requests that asked for the gradient, and scatters the results into each
 * request's own buffers.  Two waves can be in flight at once.  The launch
 * shape is fixed by ccm_serve_start from the geometry resident at that moment,
 * so a request's results are bitwise the same whatever else shares its wave.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t max_wave_pairs;      /* pairs per wave (and largest request); 0 = the
                                  most that the context's HBM budget holds */
  int64_t max_wave_requests;   /* requests per wave */
  int64_t max_queued;          /* queued (not yet running) requests */
  ccm_params params;           /* parameters of every request */
  ccm_tuning tuning;           /* launch shape (raised to the resident pieces) */
} ccm_serve_config;

/* Defaults: 16384 pairs and 1024 requests per wave, 65536 queued requests,
 * ccm_default_params, the default tuning. */
CCM_API void ccm_default_serve_config(ccm_serve_config* cfg);

/* Starts the scheduler of `ctx`: allocates two sets of wave buffers (device
 * and pinned host), captures one graph per set and starts the scheduler
 * thread.  Synchronous.  Bodies loaded later may be requested if no piece of
 * theirs has more vertices, planes or edges than the largest resident at start.
 * Device memory: two sets of wave buffers of 168 bytes per pair, 112 per
 * work item and 168 per output group, which must fit the context's HBM budget.
 * Errors: CCM_ERR_INVALID (already started, bad capacities or params, no
 * resident geometry), CCM_ERR_OOM (the wave buffers do
 * not fit the context's HBM budget or cudaMalloc failed), CCM_ERR_CUDA. */
CCM_API ccm_status ccm_serve_start(ccm_ctx ctx, const ccm_serve_config* cfg);

/* Runs every queued request to completion, stops the thread and frees the
 * wave buffers; tickets not yet polled become unknown.  ccm_destroy does the
 * same.  Errors: CCM_ERR_INVALID (not started). */
CCM_API ccm_status ccm_serve_stop(ccm_ctx ctx);

/* One request: the contacts of n_pairs body pairs (A[i], B[i]).
 *   A, B    host arrays of n_pairs handles, read before ccm_submit returns;
 *   pose_a, pose_b  device [n_pairs, 12] float32, holding their values when
 *           ccm_submit is called (synchronize the producing stream first);
 *   y       device [G, 8] float32 outputs, G = ccm_output_size of the pairs;
 *   ybar    device [G, 8] float32 cotangent, or NULL for the forward pass only;
 *   grad    device [n_pairs, 12] float32 gradient of <ybar, y> in the twist
 *           chart (w_A, v_A, w_B, v_B); required with ybar, else ignored.
 * The device buffers stay owned by the caller and must stay valid and
 * untouched until ccm_poll reports the ticket done. */
typedef struct {
  int64_t n_pairs;
  const ccm_geom* A;
  const ccm_geom* B;
  const float* pose_a;
  const float* pose_b;
  float* y;
  const float* ybar;
  float* grad;
} ccm_request;

/* Queues a request; never blocks on the GPU.  *ticket identifies it for
 * ccm_poll.  Errors: CCM_ERR_INVALID (not started, bad request or handle, a
 * body with a piece larger than the start-time launch shape holds),
 * CCM_ERR_OOM (request larger than a wave), CCM_ERR_BUSY (queue full: retry
 * after polling), CCM_ERR_CUDA (an earlier wave failed). */
CCM_API ccm_status ccm_submit(ccm_ctx ctx, const ccm_request* req, ccm_ticket* ticket);

/* Non-blocking.  *done = 1 once the request's outputs are in its buffers
 * (visible to any stream), after which the ticket is retired; *latency_s
 * (optional) then receives submit-to-completion time in seconds as seen by the
 * scheduler.  *done = 0 while it is queued or running.  Errors:
 * CCM_ERR_INVALID, CCM_ERR_UNKNOWN_TICKET (never issued or already retired),
 * CCM_ERR_CUDA (a wave failed). */
CCM_API ccm_status ccm_poll(ccm_ctx ctx, ccm_ticket ticket, int* done, double* latency_s);

/* Non-blocking completion queue: retires up to `capacity` completed requests
 * in completion order and writes their tickets (host array) and, if
 * latency_s != NULL, their submit-to-completion times in seconds; *n gets how
 * many.  Tickets already retired by ccm_poll are skipped.  Errors:
 * CCM_ERR_INVALID, CCM_ERR_CUDA (a wave failed). */
CCM_API ccm_status ccm_poll_completed(ccm_ctx ctx, ccm_ticket* tickets, double* latency_s,
                                      int64_t capacity, int64_t* n);

/* hold != 0: queued requests form no new wave until called with hold = 0
 * (waves already running finish).  ccm_serve_stop releases a hold.
 * Errors: CCM_ERR_INVALID (not started). */
CCM_API ccm_status ccm_serve_hold(ccm_ctx ctx, int hold);

/* Counters since ccm_serve_start (tracing of the serving loop). */
typedef struct {
  int64_t waves;        /* waves launched */
  int64_t served;       /* requests completed */
  int64_t wave_pairs;   /* body pairs run, summed over waves */
  int64_t wave_items;   /* work items run, summed over waves */
  double gpu_s;         /* device time of the finished waves' graphs (CUDA events) */
  double form_s;        /* host time spent forming waves (tables, order, copies) */
} ccm_serve_counters;
/* Errors: CCM_ERR_INVALID (not started). */
CCM_API ccm_status ccm_serve_stats(ccm_ctx ctx, ccm_serve_counters* out);

/* Load generator for measuring the serving loop without a client in the way:
 * on the calling thread, submits reqs[k] (host array of n requests) when
 * arrival_s[k] seconds (non-decreasing, host array) have passed since the
 * call began -- busy-waiting on a steady clock, retrying after draining when
 * the queue answers CCM_ERR_BUSY -- and drains completions with
 * ccm_poll_completed until all n are done.  Writes, per request (host arrays,
 * may be NULL), lag_s[k] = submission time - arrival time (the generator's own
 * delay) and latency_s[k] = completion - arrival as the host sees it; *elapsed_s
 * (may be NULL) gets the time from the call's start to the last completion.
 * The requests' buffers must stay valid until the call returns.  Requires a
 * started serving loop; blocks until every request is done.  The paper has no
 * counterpart: this only measures the loop.  Errors: those of ccm_submit and
 * ccm_poll_completed (requests submitted before an error still complete in
 * the loop). */
CCM_API ccm_status ccm_serve_replay(ccm_ctx ctx, const ccm_request* reqs,
                                    const double* arrival_s, int64_t n, double* lag_s,
                                    double* latency_s, double* elapsed_s);

#ifdef __cplusplus
}
#endif
#endif /* CCM_H_ */
