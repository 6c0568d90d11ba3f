/*
 * tb.h -- C ABI of the GB300 implementation of the data-parallel core of
 *   R. Levien, "Fast GPU bounding boxes on tree-structured scenes"
 *   (arXiv 2205.11659).
 *
 * A scene is a flattened tree (Sec. 1.1): a node with children is an open
 * element, its children's encoding, then a close element.  Element kinds are
 * one byte each:
 *
 *   TB_LEAF = 0        a leaf with a box
 *   TB_OPEN_CLIP = 1   opens a clip node; its box clips every descendant
 *   TB_OPEN_BLEND = 2  opens a blend node; its own box is ignored
 *   TB_CLOSE = 3       closes the innermost open node
 *
 * A box is four floats (x0, y0, x1, y1), 16 bytes, 16-byte aligned.
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Pointers named kind, box, parent, match, box_out, in, out, local,
 *    grad_world, grad_local, offsets, ws and d_status are DEVICE pointers
 *    owned by the caller.  The library allocates nothing and frees nothing.
 *  - kind and ws must be 16-byte aligned; float/float4 arrays must be
 *    16-byte aligned; int32 arrays 4-byte aligned.  Outputs must not alias
 *    inputs.
 *  - n < 2^31 (indices are int32).
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  All work is enqueued on it, nothing is synchronised, and a
 *    call can be captured into a CUDA graph.
 *  - ws is scratch of at least tb_workspace_size(op, n, num_scenes) bytes;
 *    its contents on entry do not matter.
 *  - d_status is one device int32.  The call first writes TB_OK to it in
 *    stream order, then kernels write the first data error they find
 *    (TB_ERR_UNBALANCED, TB_ERR_BAD_KIND or TB_ERR_TIMEOUT).  Read it after
 *    synchronising the stream.  When it is not TB_OK the outputs are
 *    unspecified, but every memory access stays inside the buffers above.
 *  - The return value reports argument errors found on the host before any
 *    work is enqueued (TB_ERR_INVALID_ARG, TB_ERR_WORKSPACE) or a failed
 *    launch (TB_ERR_CUDA).  n == 0 enqueues only the status write.
 */
#ifndef TB_H
#define TB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TB_OK = 0,
  TB_ERR_INVALID_ARG = 1, /* null pointer, n < 0 or too large, misalignment */
  TB_ERR_UNBALANCED = 2,  /* depth below 0 somewhere, or not 0 at the end  */
  TB_ERR_BAD_KIND = 3,    /* a kind byte above 3                           */
  TB_ERR_WORKSPACE = 4,   /* ws_bytes below tb_workspace_size()            */
  TB_ERR_TIMEOUT = 5,     /* a bounded cross-block wait gave up            */
  TB_ERR_CUDA = 6,        /* a CUDA launch or memset failed                */
  TB_ERR_BOUNDS = 7       /* debug builds only (TB_DEBUG): an index check
                             failed and the access was skipped            */
} tb_status;

enum { TB_LEAF = 0, TB_OPEN_CLIP = 1, TB_OPEN_BLEND = 2, TB_CLOSE = 3 };

/* Operations, for tb_workspace_size(). */
enum {
  TB_OP_MATCH_PARENS = 0,
  TB_OP_BBOXES = 1,
  TB_OP_BBOXES_BATCHED = 2,
  TB_OP_TREE_SCAN = 3,
  TB_OP_TREE_BACKWARD = 4,
  TB_OP_OPEN_POSITIONS = 5
};

/* Monoids and directions of tb_tree_scan. */
typedef enum {
  TB_MONOID_BBOX_ISECT = 0,   /* float4 boxes, intersection, identity (-inf,-inf,+inf,+inf) */
  TB_MONOID_BBOX_UNION = 1,   /* float4 boxes, union, identity (+inf,+inf,-inf,-inf) */
  TB_MONOID_ADD_I32 = 2,      /* int32, addition modulo 2^32, identity 0 */
  TB_MONOID_AFFINE3X4_F32 = 3, /* 12 floats, row-major [R | t] (x -> R x + t),
                                 composition A*B = apply B then A, identity [I | 0] */
  TB_MONOID_RIGID_F32 = 4      /* 8 floats (qx, qy, qz, qw, tx, ty, tz, unused): rotation
                                 by the unit quaternion q then translation t,
                                 x -> q x q* + t; composition A*B = apply B then A =
                                 (qA qB, tA + qA tB qA*) with Hamilton's product;
                                 identity (0, 0, 0, 1, 0, 0, 0, 0).  No
                                 renormalisation: rounding drifts |q| by about
                                 1e-7 per level */
} tb_monoid;

typedef enum {
  TB_DOWN = 0, /* each joint: fold along its root path, the root first */
  TB_UP = 1    /* each joint: fold over its subtree, in stream order */
} tb_dir;

/* Bytes of scratch the operation needs for n elements (num_scenes is used
 * by TB_OP_BBOXES_BATCHED only).  Never fails; 0 for n == 0. */
size_t tb_workspace_size(int op, int64_t n, int64_t num_scenes);

/* Parentheses matching, strong form (Sec. 2, Fig. 1).
 *   parent[i] = the stack top before element i is processed: the
 *               innermost enclosing open for a leaf or an open, the matching
 *               open for a close, -1 at the root.
 *   match[i]  = the matching close of an open, the matching open of a close,
 *               -1 for a leaf.
 * Computed with the bicyclic semigroup (Sec. 3) and stack slices (Sec. 4,
 * Sec. 7) in a single pass over the kind stream plus a tile-level resolve. */
tb_status tb_match_parens(const uint8_t* kind, int64_t n, int32_t* parent,
                          int32_t* match, void* ws, size_t ws_bytes,
                          int32_t* d_status, void* stream);

/* Bounding boxes over the tree (Sec. 1, Sec. 6, Sec. 9).
 *   leaf:  box_out = its box intersected with the box of every OPEN_CLIP
 *          ancestor; empty (x0 >= x1 or y0 >= y1) results are written as the
 *          canonical empty box (+inf, +inf, -inf, -inf).
 *   open and its close: box_out = union of the canonical clipped boxes of all
 *          descendant leaves (the canonical empty box if there are none).
 * parent and match are as in tb_match_parens and may be NULL to skip them.
 * box is read for LEAF and OPEN_CLIP elements only. */
tb_status tb_bboxes(const uint8_t* kind, const float* box, int64_t n,
                    int32_t* parent, int32_t* match, float* box_out, void* ws,
                    size_t ws_bytes, int32_t* d_status, void* stream);

/* tb_bboxes over num_scenes independent scenes laid end to end: scene s is
 * elements [offsets[s], offsets[s+1]) with offsets[0] = 0 and
 * offsets[num_scenes] = n_total, non-decreasing (device int64 array of
 * num_scenes + 1 entries).  Matching never crosses a scene boundary: each
 * scene must be balanced on its own (TB_ERR_UNBALANCED otherwise), and
 * parent and match are scene-local indices with -1 at each scene's roots.
 * One set of launches covers all scenes. */
tb_status tb_bboxes_batched(const uint8_t* kind, const float* box,
                            const int64_t* offsets, int64_t num_scenes,
                            int64_t n_total, int32_t* parent, int32_t* match,
                            float* box_out, void* ws, size_t ws_bytes,
                            int32_t* d_status, void* stream);

/* tb_bboxes (offsets == NULL) or tb_bboxes_batched (offsets and num_scenes
 * as there) that also writes, per element, the running clip intersection of
 * the stack snapshot (Sec. 9: each entry of the snapshot is its element's box
 * intersected with the boxes of all its clip ancestors):
 *   LEAF, OPEN_CLIP:  own box intersected with the clip in force (the
 *                     intersection of all its OPEN_CLIP ancestors' boxes);
 *   OPEN_BLEND:       the clip in force (its own box is ignored);
 *   CLOSE:            the value of the open it closes.
 * The clip in force at a root is the universe (-inf, -inf, +inf, +inf).  The
 * raw intersection is written (x0 >= x1 or y0 >= y1 when empty, not the
 * canonical empty box): it is what flows down the clip chain.  clip_out holds
 * n float4 (16-byte aligned, must not alias other buffers); it may not be
 * NULL when n > 0 (TB_ERR_INVALID_ARG).  Everything else, including the
 * workspace (tb_workspace_size(TB_OP_BBOXES, n)), is as in tb_bboxes. */
tb_status tb_bboxes_clip(const uint8_t* kind, const float* box,
                         const int64_t* offsets, int64_t num_scenes, int64_t n,
                         int32_t* parent, int32_t* match, float* box_out,
                         float* clip_out, void* ws, size_t ws_bytes,
                         int32_t* d_status, void* stream);

/* Stream compaction of the opens (Sec. 1.1: a renderer keeps just the clip
 * and blend nodes this way).  pos[r] = the stream index of the r-th open
 * (OPEN_CLIP or OPEN_BLEND) in stream order, which is the element of joint
 * r of tb_tree_scan; *d_count = the number of opens (a device int32).
 *   - pos holds max_opens int32 entries; only r < max_opens are written, so
 *     a short buffer is safe and *d_count still reports all opens (a
 *     balanced stream has at most n / 2).
 *   - Bytes above 3 are reported as TB_ERR_BAD_KIND in d_status (and counted
 *     as leaves).  Nesting is not checked: any byte stream of kinds works.
 * Results are exact and deterministic.  Reads kind twice, writes 4 bytes per
 * open. */
tb_status tb_open_positions(const uint8_t* kind, int64_t n, int32_t* pos,
                            int64_t max_opens, int32_t* d_count, void* ws,
                            size_t ws_bytes, int32_t* d_status, void* stream);

/* Tree scans: the monoid generalisation of Sec. 1 and Sec. 13 (any
 * associative operation with an identity, neither commutative nor
 * idempotent required).  Values belong to the opens ("joints"): joint r is
 * the r-th open of the stream (pre-order rank), leaves carry none.
 * num_joints must equal the number of opens (at most n / 2); in and out hold
 * num_joints values of the monoid's type (4, 16, 48 or 32 bytes each), are
 * 16-byte aligned whatever the monoid, and must not overlap.
 *   TB_DOWN: out[r] = in[root] * ... * in[parent(r)] * in[r]
 *            (ancestor on the left; for transforms, world = parent world
 *            times local).
 *   TB_UP:   out[r] = fold of in[d] over the joints d of r's subtree (r
 *            itself first), in stream order.
 * A stream of several trees (a forest, e.g. skeletons laid end to end) is
 * fine: each tree is scanned on its own.  A wrong num_joints is reported as
 * TB_ERR_INVALID_ARG in d_status; unbalanced streams and bad kinds as in
 * tb_match_parens.  tb_open_positions gives the element of every joint.
 * For a monoid other than these four, tb_monoid.cuh (next to this header)
 * instantiates the same scans for a caller-defined type. */
tb_status tb_tree_scan(int monoid, int dir, const uint8_t* kind, int64_t n,
                       int64_t num_joints, const void* in, void* out, void* ws,
                       size_t ws_bytes, int32_t* d_status, void* stream);

/* Adjoint of the affine TB_DOWN scan for the loss sum_r <W_r, world_r>
 * (Frobenius product of 3x4 matrices), given grad_world[r] = W_r:
 *   grad_local[r] = d loss / d local[r]
 * local, grad_world and grad_local hold num_joints 3x4 row-major float
 * matrices.  The forward transforms are recomputed, not read from a saved
 * forward pass.  With A_r = sum over r's subtree of W_d (x) world_d^T (the
 * product of homogeneous 4x4 forms), Gbar_r = A_r world_r^{-T} and
 * grad_local[r] = R_parent(r)^T Gbar_r (Gbar_r at a root), where R is the
 * rotation part of the parent's world transform.  Needs invertible local
 * rotation parts. */
tb_status tb_tree_scan_affine_backward(const uint8_t* kind, int64_t n,
                                       int64_t num_joints, const float* local,
                                       const float* grad_world,
                                       float* grad_local, void* ws,
                                       size_t ws_bytes, int32_t* d_status,
                                       void* stream);

/* tb_tree_scan_affine_backward after a scan of the same stream: the joint
 * structure (joint depths, parents and subtree ends) is read from ws instead
 * of being computed again; the forward transforms are still recomputed.
 * ws (at least tb_workspace_size(TB_OP_TREE_BACKWARD, n) bytes) must hold
 * what the last tb_tree_scan(..., TB_DOWN or TB_UP, ...) or
 * tb_tree_scan_affine_backward call that used it left there, for this kind
 * stream, n and num_joints, with nothing else writing ws in between.  That
 * call records n and num_joints in ws once the structure is complete (its
 * d_status TB_OK); when they differ, or that call failed, this call reports
 * TB_ERR_INVALID_ARG in d_status and writes no gradients.  A different kind
 * stream of the same n and num_joints is not detected and gives wrong
 * gradients (every memory access stays inside the buffers all the same).
 * Arguments and results otherwise as tb_tree_scan_affine_backward.  No paper
 * counterpart: the reuse an autograd pair (forward, then its backward) can
 * make of the forward's workspace. */
tb_status tb_tree_scan_affine_backward_reuse(const uint8_t* kind, int64_t n,
                                             int64_t num_joints, const float* local,
                                             const float* grad_world,
                                             float* grad_local, void* ws,
                                             size_t ws_bytes, int32_t* d_status,
                                             void* stream);

/* Joint-level structure of the tree the kind stream describes: the depth,
 * parent and left-sibling vectors (the paper relates parentheses matching
 * to deriving parent and left-sibling vectors from a depth vector, Sec. 12).
 * Joint r is the r-th open of the stream (pre-order).  For every joint:
 *   depth_out[r]         1 at a root, one more than its parent otherwise;
 *   parent_out[r]        the parent joint, -1 at a root;
 *   left_sibling_out[r]  the previous joint with the same parent, -1 for a
 *                        first child (the roots of a forest are siblings).
 * Each output is a device array of num_joints int32, or NULL to skip it.
 * num_joints must be the number of opens in the stream (else
 * TB_ERR_INVALID_ARG in d_status).  ws: at least
 * tb_workspace_size(TB_OP_TREE_SCAN, n) bytes.  Errors of the stream are
 * reported in d_status as for tb_tree_scan; the outputs are then undefined. */
tb_status tb_tree_structure(const uint8_t* kind, int64_t n, int64_t num_joints,
                            int32_t* depth_out, int32_t* parent_out,
                            int32_t* left_sibling_out, void* ws, size_t ws_bytes,
                            int32_t* d_status, void* stream);

/* Tracing hook.  After tb_set_phase_events(events, k) (1 <= k <= 16) every
 * later call on this host thread records, on its own stream, events[0],
 * events[1], ... in launch order: one before each kernel of the call and
 * one after its last kernel, until the k events run out.  The matching
 * calls (tb_match_parens, tb_bboxes, tb_bboxes_batched) use five: before the
 * tile-summary pass, the tile-level resolve, the main tile pass and the
 * cross-tile union step, and at the end.  The tree calls record one before
 * each of their kernels (depth pass, tile minima, min tree over the tiles,
 * structure pass, then the scan's own kernels) and one at the end.  events
 * holds cudaEvent_t handles created by the
 * caller; tb_set_phase_events(NULL, 0) turns the hook off. */
tb_status tb_set_phase_events(void* const* events, int num_events);

/* Allocation-free form of tb_bboxes, for callers that cannot allocate
 * device memory: code that must not call cudaMalloc while it runs (a
 * renderer's per-frame path or a real-time loop with a fixed memory budget,
 * a plug-in whose host application owns all device memory, work issued
 * where allocation would synchronise the device).  The paper has no
 * counterpart; it is an interface convenience.
 *
 * Same results as tb_bboxes, but the scratch is a file-scope device array of
 * the library (5 MiB, held by every GPU that loads the library until the
 * process exits), so there is no ws argument.  The caller still passes the
 * inputs and outputs (d_status included).
 *  - n may be at most TB_STATIC_WS_MAX_N; larger n returns TB_ERR_WORKSPACE
 *    and a negative n TB_ERR_INVALID_ARG, without enqueuing anything.
 *  - The first call on each device looks up that device's address of the
 *    array (cudaGetSymbolAddress, with that device current); make that first
 *    call before any stream capture.  It allocates nothing, now or later.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; each call clears what must start at zero.  Calls whose work
 *    overlaps on the GPU (other streams, other host threads) race on the
 *    array and give wrong results: keep them ordered on one stream. */
#define TB_STATIC_WS_MAX_N (1 << 17)
tb_status tb_bboxes_static_ws(const uint8_t* kind, const float* box, int64_t n,
                              int32_t* parent, int32_t* match, float* box_out,
                              int32_t* d_status, void* stream);

/* Test hook for the bounded cross-block waits (failure detection): after
 * tb_debug_withhold_tile(t), element tile t (4096 elements each) of the
 * depth pass of the following tb_tree_scan / tb_tree_scan_affine_backward
 * calls on this host thread never publishes its look-back word, so the
 * tiles after it give up after about a second and the call reports
 * TB_ERR_TIMEOUT in d_status; the later kernels then stop and the outputs
 * are unspecified, and the CUDA context stays usable.  The matching and
 * bounding-box calls have no cross-block wait and ignore the hook.  -1
 * turns the hook off; values below -1 return TB_ERR_INVALID_ARG.  The paper
 * has no counterpart. */
tb_status tb_debug_withhold_tile(int tile);

/* Library version string. */
const char* tb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TB_H */
