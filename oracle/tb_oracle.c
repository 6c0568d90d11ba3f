/*
 * tb_oracle.c -- plain sequential CPU oracle for the method of
 *   R. Levien, "Fast GPU bounding boxes on tree-structured scenes"
 *   (arXiv 2205.11659).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the timed
 * CPU baseline of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA path and never calls it.  Every function is
 * the paper's sequential definition written out directly, in stream order,
 * with one stack and no blocking, fusion or reordering:
 *
 *   orc_bic                 -- Sec. 3, the bicyclic semigroup reduction
 *   orc_stack_slice         -- Sec. 4, the stack monoid Stk(enum(s))
 *   orc_match_parens        -- Sec. 2 / Fig. 1, the strong matching problem
 *   orc_bboxes              -- Sec. 1 and Sec. 6: clip = intersection flowing
 *                              down, blend = union flowing up
 *   orc_bboxes_batched      -- orc_bboxes per scene, scene-local indices
 *   orc_clip_out            -- Sec. 9, the stack snapshot's running clip
 *                              intersection, per element
 *   orc_open_positions      -- Sec. 1.1, stream compaction of the clip and
 *                              blend nodes (the opens), in stream order
 *   orc_tree_scan_*         -- Sec. 1 / Sec. 13, "any monoid" over the tree
 *   orc_affine_*            -- the same stack walk for 3x4 affine transforms
 *                              (root-path products) and their adjoint, fp64
 *   orc_rigid_scan          -- the same for rigid transforms (unit quaternion
 *                              and translation), DOWN and UP, fp64
 *   orc_tree_structure      -- the joint-level depth, parent and left-sibling
 *                              vectors (Sec. 12 relates the matching to parent
 *                              and left-sibling vectors of a depth vector)
 *
 * Element kinds: 0 = LEAF, 1 = OPEN_CLIP, 2 = OPEN_BLEND, 3 = CLOSE.
 * A box is 4 floats (x0, y0, x1, y1).
 *
 * Readings where the paper is silent (listed again in the design notes):
 *  - parent of a CLOSE is its matching open (Fig. 1 prints the stack top
 *    before the element); match of a LEAF is -1; root parent is -1.
 *  - a stream whose running depth goes below 0 or ends above 0 is an error
 *    (status 2); a kind above 3 is an error (status 3).
 *  - intersection identity is (-inf,-inf,+inf,+inf); union identity and the
 *    canonical empty box are (+inf,+inf,-inf,-inf); a box is empty when
 *    x0 >= x1 or y0 >= y1; a leaf's clipped box is made canonical before it
 *    enters any union; the raw (possibly empty) intersection is what flows
 *    down the clip chain.
 *  - a blend node's own box is ignored; every OPEN (clip or blend) gets the
 *    union of its descendant leaves, written at its open and its close.
 *
 * Precision: min/max of fp32 values is exact, so the box results here are
 * the exact results of the definitions, independent of evaluation order.
 * The transform functions use fp64 throughout.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_UNBALANCED 2
#define ORC_BAD_KIND 3

enum { K_LEAF = 0, K_OPEN_CLIP = 1, K_OPEN_BLEND = 2, K_CLOSE = 3 };

static int is_open(uint8_t k) { return k == K_OPEN_CLIP || k == K_OPEN_BLEND; }

static int check_kinds(const uint8_t* kind, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (kind[i] > 3) return ORC_BAD_KIND;
  return ORC_OK;
}

/* ---------------------------------------------------------------- Sec. 3 */
/* Bicyclic semigroup: (a,b) + (c,d) = (a + c - min(b,c), b + d - min(b,c)).
 * An open maps to (0,1), a close to (1,0); a leaf is the identity (0,0). */
void orc_bic_combine(int64_t a, int64_t b, int64_t c, int64_t d,
                     int64_t* ra, int64_t* rb) {
  int64_t m = b < c ? b : c;
  *ra = a + c - m;
  *rb = b + d - m;
}

int orc_bic(const uint8_t* kind, int64_t n, int64_t* out_a, int64_t* out_b) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t a = 0, b = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t ea = 0, eb = 0;
    if (is_open(kind[i])) eb = 1;
    else if (kind[i] == K_CLOSE) ea = 1;
    orc_bic_combine(a, b, ea, eb, &a, &b);
  }
  *out_a = a;
  *out_b = b;
  return ORC_OK;
}

/* ---------------------------------------------------------------- Sec. 4 */
/* Stack monoid over enum(s): (a0,l0) + (a1,l1) =
 *   (a0 + a1 - min(|l0|,a1), l0[..max(0,|l0|-a1)] ++ l1).
 * Folded left to right one element at a time: an open at index i is
 * (0,[i]), a close is (1,[]), a leaf is (0,[]).  Writes the list (bottom of
 * the stack first) to list_out and returns its length; *a_out receives the
 * count of unmatched closes. */
int64_t orc_stack_slice(const uint8_t* kind, int64_t n, int64_t* a_out,
                        int64_t* list_out) {
  int64_t a = 0, len = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (is_open(kind[i])) {
      /* (a,l) + (0,[i]) */
      list_out[len++] = i;
    } else if (kind[i] == K_CLOSE) {
      /* (a,l) + (1,[]) */
      int64_t m = len < 1 ? len : 1;
      a = a + 1 - m;
      len = len - m;
    }
  }
  *a_out = a;
  return len;
}

/* ------------------------------------------------------- Sec. 2, Fig. 1 */
/* Strong matching problem: for every element the stack top before it is
 * processed (its enclosing open; for a close, the open it matches), and the
 * classical match (open <-> close, -1 for a leaf).  The paper's sentinel -1
 * at the stack bottom is the root value. */
int orc_match_parens(const uint8_t* kind, int64_t n, int32_t* parent,
                     int32_t* match) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t sp = 0;
  st = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    parent[i] = sp > 0 ? (int32_t)stack[sp - 1] : -1;
    match[i] = -1;
    if (is_open(kind[i])) {
      stack[sp++] = i;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      int64_t o = stack[--sp];
      match[i] = (int32_t)o;
      match[o] = (int32_t)i;
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(stack);
  return st;
}

/* ------------------------------------------------------------ Sec. 1.1 */
/* Stream compaction of the opens: the index of every OPEN_CLIP or
 * OPEN_BLEND element, in stream order (so entry r is the element of the
 * r-th open, joint r of the tree scans).  Entries r < cap are written;
 * *count receives the number of opens.  Nesting is not checked. */
int orc_open_positions(const uint8_t* kind, int64_t n, int32_t* pos, int64_t cap,
                       int64_t* count) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t r = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (is_open(kind[i])) {
      if (r < cap) pos[r] = (int32_t)i;
      ++r;
    }
  }
  *count = r;
  return ORC_OK;
}

/* ------------------------------------------------------ Sec. 1, Sec. 6 */
static void box_isect(const float* a, const float* b, float* r) {
  r[0] = a[0] > b[0] ? a[0] : b[0];
  r[1] = a[1] > b[1] ? a[1] : b[1];
  r[2] = a[2] < b[2] ? a[2] : b[2];
  r[3] = a[3] < b[3] ? a[3] : b[3];
}
static void box_union(const float* a, const float* b, float* r) {
  r[0] = a[0] < b[0] ? a[0] : b[0];
  r[1] = a[1] < b[1] ? a[1] : b[1];
  r[2] = a[2] > b[2] ? a[2] : b[2];
  r[3] = a[3] > b[3] ? a[3] : b[3];
}
static void box_set(float* r, float x0, float y0, float x1, float y1) {
  r[0] = x0; r[1] = y0; r[2] = x1; r[3] = y1;
}
static void box_canon(float* r) {
  if (r[0] >= r[2] || r[1] >= r[3])
    box_set(r, INFINITY, INFINITY, -INFINITY, -INFINITY);
}

typedef struct {
  int64_t open;   /* index of the open element */
  float clip[4];  /* intersection of the clip boxes on the root path */
  float uni[4];   /* union of the clipped leaves seen inside so far */
} orc_entry;

/* The sequential algorithm of Sec. 1: walk the flattened tree keeping a
 * stack whose entries carry one box for clipping and one for blending.  A
 * leaf is intersected with the clip accumulated on its root path (Sec. 6.1
 * definition); a node receives the union of its descendant leaves (Sec. 6.2
 * definition), produced at the close and written to the open as well. */
int orc_bboxes(const uint8_t* kind, const float* box, int64_t n,
               int32_t* parent, int32_t* match, float* box_out) {
  int st = check_kinds(kind, n);
  if (st) return st;
  orc_entry* stack = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)(n + 1));
  int64_t sp = 0;
  float universe[4] = {-INFINITY, -INFINITY, INFINITY, INFINITY};
  st = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    const float* cur = sp > 0 ? stack[sp - 1].clip : universe;
    if (parent) parent[i] = sp > 0 ? (int32_t)stack[sp - 1].open : -1;
    if (match) match[i] = -1;
    const float* bi = box + 4 * i;
    float* oi = box_out + 4 * i;
    switch (kind[i]) {
      case K_LEAF: {
        box_isect(bi, cur, oi);
        box_canon(oi);
        if (sp > 0) box_union(stack[sp - 1].uni, oi, stack[sp - 1].uni);
        break;
      }
      case K_OPEN_CLIP:
      case K_OPEN_BLEND: {
        orc_entry* e = &stack[sp];
        e->open = i;
        if (kind[i] == K_OPEN_CLIP) box_isect(bi, cur, e->clip);
        else memcpy(e->clip, cur, sizeof(e->clip));
        box_set(e->uni, INFINITY, INFINITY, -INFINITY, -INFINITY);
        ++sp;
        break;
      }
      case K_CLOSE: {
        if (sp == 0) { st = ORC_UNBALANCED; goto done; }
        orc_entry* e = &stack[--sp];
        if (match) { match[i] = (int32_t)e->open; match[e->open] = (int32_t)i; }
        memcpy(oi, e->uni, sizeof(e->uni));
        memcpy(box_out + 4 * e->open, e->uni, sizeof(e->uni));
        if (sp > 0) box_union(stack[sp - 1].uni, e->uni, stack[sp - 1].uni);
        break;
      }
    }
  }
  if (sp != 0) st = ORC_UNBALANCED;
done:
  free(stack);
  return st;
}

/* The clip value of the stack snapshot at every element (Sec. 9: each
 * entry is the intersection of its element's box with the boxes of all its
 * clip ancestors).  LEAF and OPEN_CLIP: own box intersected with the clip in
 * force; OPEN_BLEND: the clip in force (its box is ignored); CLOSE: the value
 * of the open it closes.  The raw intersection is written, not made
 * canonical (it is what flows down the clip chain).  Root clip: universe. */
int orc_clip_out(const uint8_t* kind, const float* box, int64_t n, float* clip_out) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t sp = 0;
  float universe[4] = {-INFINITY, -INFINITY, INFINITY, INFINITY};
  st = ORC_OK;
  for (int64_t i = 0; i < n; ++i) {
    const float* cur = sp > 0 ? clip_out + 4 * stack[sp - 1] : universe;
    float* oi = clip_out + 4 * i;
    switch (kind[i]) {
      case K_LEAF:
      case K_OPEN_CLIP:
        box_isect(box + 4 * i, cur, oi);
        if (kind[i] == K_OPEN_CLIP) stack[sp++] = i;
        break;
      case K_OPEN_BLEND:
        memcpy(oi, cur, 4 * sizeof(float));
        stack[sp++] = i;
        break;
      case K_CLOSE:
        if (sp == 0) { st = ORC_UNBALANCED; goto done; }
        memcpy(oi, clip_out + 4 * stack[--sp], 4 * sizeof(float));
        break;
    }
  }
  if (sp != 0) st = ORC_UNBALANCED;
done:
  free(stack);
  return st;
}

/* Many independent scenes laid end to end; scene s covers
 * [offsets[s], offsets[s+1]).  Each is solved on its own, and parent/match
 * are scene-local.  The first failing scene's status is returned. */
int orc_bboxes_batched(const uint8_t* kind, const float* box,
                       const int64_t* offsets, int64_t num_scenes,
                       int32_t* parent, int32_t* match, float* box_out) {
  for (int64_t s = 0; s < num_scenes; ++s) {
    int64_t b = offsets[s], e = offsets[s + 1];
    int st = orc_bboxes(kind + b, box + 4 * b, e - b, parent ? parent + b : NULL,
                        match ? match + b : NULL, box_out + 4 * b);
    if (st) return st;
  }
  return ORC_OK;
}

/* ------------------------------------------- Sec. 1 / Sec. 13: monoids */
/* Values are given per OPEN in pre-order (the order opens appear in the
 * stream); leaves carry none.  DOWN gives each open the fold along its root
 * path, ancestor first.  UP gives each open the fold of its own value and
 * all its descendants' values, in stream order. */
#define ORC_DOWN 0
#define ORC_UP 1

int orc_tree_scan_i32(int dir, const uint8_t* kind, int64_t n,
                      const int32_t* in, int32_t* out) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t* acc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  int64_t sp = 0, r = 0;
  for (int64_t i = 0; i < n && st == ORC_OK; ++i) {
    if (is_open(kind[i])) {
      int32_t v = in[r];
      if (dir == ORC_DOWN) {
        acc[sp] = sp > 0 ? acc[sp - 1] + v : v;
        out[r] = acc[sp];
      } else {
        acc[sp] = v;
      }
      rank[sp++] = r++;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      --sp;
      if (dir == ORC_UP) {
        out[rank[sp]] = acc[sp];
        if (sp > 0) acc[sp - 1] = acc[sp - 1] + acc[sp];
      }
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(rank);
  free(acc);
  return st;
}

/* Joint r is the r-th open.  depth[r] = the number of opens enclosing it
 * plus one; parent[r] = the joint of the enclosing open, -1 at a root;
 * left_sibling[r] = the previous joint with the same parent (roots are the
 * children of one virtual root), -1 for a first child.  Any output may be
 * NULL. */
int orc_tree_structure(const uint8_t* kind, int64_t n, int32_t* depth, int32_t* parent,
                       int32_t* left_sibling) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* joint = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));     /* joint on the stack */
  int64_t* lastc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 2));     /* last child per level */
  int64_t sp = 0, r = 0;
  lastc[0] = -1;
  for (int64_t i = 0; i < n; ++i) {
    if (is_open(kind[i])) {
      if (depth) depth[r] = (int32_t)(sp + 1);
      if (parent) parent[r] = sp > 0 ? (int32_t)joint[sp - 1] : -1;
      if (left_sibling) left_sibling[r] = (int32_t)lastc[sp];
      lastc[sp] = r;
      joint[sp++] = r++;
      lastc[sp] = -1;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      --sp;
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(joint);
  free(lastc);
  return st;
}

/* monoid 0: intersection, monoid 1: union (both on raw boxes, no canon). */
int orc_tree_scan_box(int monoid, int dir, const uint8_t* kind, int64_t n,
                      const float* in, float* out) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  float* acc = (float*)malloc(sizeof(float) * 4 * (size_t)(n + 1));
  int64_t sp = 0, r = 0;
  for (int64_t i = 0; i < n && st == ORC_OK; ++i) {
    if (is_open(kind[i])) {
      const float* v = in + 4 * r;
      float* a = acc + 4 * sp;
      if (dir == ORC_DOWN && sp > 0) {
        if (monoid == 0) box_isect(acc + 4 * (sp - 1), v, a);
        else box_union(acc + 4 * (sp - 1), v, a);
      } else {
        memcpy(a, v, 4 * sizeof(float));
      }
      if (dir == ORC_DOWN) memcpy(out + 4 * r, a, 4 * sizeof(float));
      rank[sp++] = r++;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      --sp;
      if (dir == ORC_UP) {
        memcpy(out + 4 * rank[sp], acc + 4 * sp, 4 * sizeof(float));
        if (sp > 0) {
          if (monoid == 0) box_isect(acc + 4 * (sp - 1), acc + 4 * sp, acc + 4 * (sp - 1));
          else box_union(acc + 4 * (sp - 1), acc + 4 * sp, acc + 4 * (sp - 1));
        }
      }
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(rank);
  free(acc);
  return st;
}

/* ------------------------------------------------ 3x4 affine transforms */
/* A transform is 12 doubles, row-major [R | t] (3 rows of r r r t), acting
 * on column vectors: x -> R x + t.  Composition (A*B) = [RA RB | RA tB + tA]:
 * B is applied first, so A*B with A the ancestor puts the ancestor on the
 * left. */
static void aff_mul(const double* A, const double* B, double* C) {
  double T[12];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[4 * r + k] * B[4 * k + c];
      T[4 * r + c] = s;
    }
    double s = A[4 * r + 3];
    for (int k = 0; k < 3; ++k) s += A[4 * r + k] * B[4 * k + 3];
    T[4 * r + 3] = s;
  }
  memcpy(C, T, sizeof(T));
}

/* Forward: world_r = world_parent(r) * L_r for every joint r (an OPEN, in
 * pre-order); a root's world is its local transform.  Optionally reports
 * each joint's parent joint (-1 at a root). */
static int affine_forward_impl(const uint8_t* kind, int64_t n, const double* local,
                               double* world, int64_t* parent_joint) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t sp = 0, r = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (is_open(kind[i])) {
      if (sp > 0) aff_mul(world + 12 * stack[sp - 1], local + 12 * r, world + 12 * r);
      else memcpy(world + 12 * r, local + 12 * r, 12 * sizeof(double));
      if (parent_joint) parent_joint[r] = sp > 0 ? stack[sp - 1] : -1;
      stack[sp++] = r++;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      --sp;
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(stack);
  return st;
}

int orc_affine_forward(const uint8_t* kind, int64_t n, const double* local,
                       double* world) {
  return affine_forward_impl(kind, n, local, world, NULL);
}

/* UP over affine transforms: each joint receives the product, in stream
 * order, of its own transform and those of all its descendants. */
int orc_affine_up(const uint8_t* kind, int64_t n, const double* in, double* out) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  double* acc = (double*)malloc(sizeof(double) * 12 * (size_t)(n + 1));
  int64_t sp = 0, r = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (is_open(kind[i])) {
      memcpy(acc + 12 * sp, in + 12 * r, 12 * sizeof(double));
      rank[sp++] = r++;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      --sp;
      memcpy(out + 12 * rank[sp], acc + 12 * sp, 12 * sizeof(double));
      if (sp > 0) aff_mul(acc + 12 * (sp - 1), acc + 12 * sp, acc + 12 * (sp - 1));
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(rank);
  free(acc);
  return st;
}

/* ------------------------------------- rigid transforms (quaternion, t) */
/* A rigid transform is 8 doubles (qx, qy, qz, qw, tx, ty, tz, unused): a
 * rotation by the unit quaternion q = w + xi + yj + zk, then a translation:
 * x -> q x q* + t.  Composition (A*B) = (qA qB, tA + qA tB qA*): B first, so
 * the ancestor is on the left as for the affine transforms (Sec. 1 and
 * Sec. 13: any monoid).  Quaternions multiply by Hamilton's rules
 * i^2 = j^2 = k^2 = ijk = -1. */
static void quat_mul(const double* a, const double* b, double* c) {
  const double ax = a[0], ay = a[1], az = a[2], aw = a[3];
  const double bx = b[0], by = b[1], bz = b[2], bw = b[3];
  c[0] = aw * bx + ax * bw + ay * bz - az * by;
  c[1] = aw * by - ax * bz + ay * bw + az * bx;
  c[2] = aw * bz + ax * by - ay * bx + az * bw;
  c[3] = aw * bw - ax * bx - ay * by - az * bz;
}

/* v rotated by q: q v q* with v a pure quaternion. */
static void quat_rotate(const double* q, const double* v, double* out) {
  const double p[4] = {v[0], v[1], v[2], 0.0};
  const double qc[4] = {-q[0], -q[1], -q[2], q[3]};
  double t[4], r[4];
  quat_mul(q, p, t);
  quat_mul(t, qc, r);
  out[0] = r[0];
  out[1] = r[1];
  out[2] = r[2];
}

static void rigid_mul(const double* A, const double* B, double* C) {
  double q[4], t[3];
  quat_mul(A, B, q);
  quat_rotate(A, B + 4, t);
  C[0] = q[0];
  C[1] = q[1];
  C[2] = q[2];
  C[3] = q[3];
  C[4] = A[4] + t[0];
  C[5] = A[5] + t[1];
  C[6] = A[6] + t[2];
  C[7] = 0.0;
}

/* DOWN (dir 0): each joint gets the product along its root path, the root
 * first; UP (dir 1): the product over its subtree in stream order, its own
 * value first.  Same stack walks as the affine forms above. */
int orc_rigid_scan(int dir, const uint8_t* kind, int64_t n, const double* in, double* out) {
  int st = check_kinds(kind, n);
  if (st) return st;
  int64_t* stack = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  double* acc = (double*)malloc(sizeof(double) * 8 * (size_t)(n + 1));
  int64_t sp = 0, r = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (is_open(kind[i])) {
      if (dir == 0) {
        if (sp > 0) rigid_mul(out + 8 * stack[sp - 1], in + 8 * r, out + 8 * r);
        else memcpy(out + 8 * r, in + 8 * r, 8 * sizeof(double));
      } else {
        memcpy(acc + 8 * sp, in + 8 * r, 8 * sizeof(double));
      }
      stack[sp++] = r++;
    } else if (kind[i] == K_CLOSE) {
      if (sp == 0) { st = ORC_UNBALANCED; break; }
      --sp;
      if (dir != 0) {
        memcpy(out + 8 * stack[sp], acc + 8 * sp, 8 * sizeof(double));
        if (sp > 0) rigid_mul(acc + 8 * (sp - 1), acc + 8 * sp, acc + 8 * (sp - 1));
      }
    }
  }
  if (st == ORC_OK && sp != 0) st = ORC_UNBALANCED;
  free(stack);
  free(acc);
  return st;
}

/* loss = sum over joints of <W_r, world_r> (Frobenius product of 3x4). */
int orc_affine_loss(const uint8_t* kind, int64_t n, const double* local,
                    const double* W, int64_t num_joints, double* loss) {
  double* world = (double*)malloc(sizeof(double) * 12 * (size_t)(num_joints + 1));
  int st = affine_forward_impl(kind, n, local, world, NULL);
  double s = 0.0;
  for (int64_t r = 0; r < num_joints * 12; ++r) s += W[r] * world[r];
  *loss = s;
  free(world);
  return st;
}

/* Adjoint of the forward map for loss = sum <W_r, world_r>.
 * world_c = world_p * L_c, so the gradient reaching world_p from a child c is
 * Gbar_c (x) L_c^T = [Gbar_c^R R_c^T + Gbar_c^t t_c^T | Gbar_c^t], and
 * Gbar_r = W_r + sum over children.  Children follow their parent in
 * pre-order, so visiting joints in reverse pre-order completes every Gbar
 * before it is used.  dL_r = R_parent^T Gbar_r (Gbar_r itself at a root). */
int orc_affine_backward(const uint8_t* kind, int64_t n, const double* local,
                        const double* grad_world, double* grad_local,
                        int64_t num_joints) {
  double* world = (double*)malloc(sizeof(double) * 12 * (size_t)(num_joints + 1));
  double* gbar = (double*)malloc(sizeof(double) * 12 * (size_t)(num_joints + 1));
  int64_t* pj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(num_joints + 1));
  int st = affine_forward_impl(kind, n, local, world, pj);
  if (st == ORC_OK) {
    memcpy(gbar, grad_world, sizeof(double) * 12 * (size_t)num_joints);
    for (int64_t c = num_joints - 1; c >= 0; --c) {
      const double* G = gbar + 12 * c;
      const double* L = local + 12 * c;
      int64_t p = pj[c];
      if (p >= 0) {
        double* Gp = gbar + 12 * p;
        for (int r = 0; r < 3; ++r) {
          for (int col = 0; col < 3; ++col) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += G[4 * r + k] * L[4 * col + k];
            s += G[4 * r + 3] * L[4 * col + 3];
            Gp[4 * r + col] += s;
          }
          Gp[4 * r + 3] += G[4 * r + 3];
        }
        const double* Wp = world + 12 * p; /* R_parent = rotation part of world_p */
        double* D = grad_local + 12 * c;
        for (int r = 0; r < 3; ++r)
          for (int col = 0; col < 4; ++col) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Wp[4 * k + r] * G[4 * k + col];
            D[4 * r + col] = s;
          }
      } else {
        memcpy(grad_local + 12 * c, G, 12 * sizeof(double));
      }
    }
  }
  free(world);
  free(gbar);
  free(pj);
  return st;
}
