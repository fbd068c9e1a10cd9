/*
 * "structure": a spring mesh that cracks under load -- oracle (test
 * infrastructure only; never linked into the CUDA library).
 *
 * Follows the thesis' finite-element application (Sec. 7.4): nodes of three
 * kinds (anchor nodes are fixed, pull nodes move with a constant velocity,
 * ordinary nodes move under the spring forces), each with up to three
 * springs; a spring pulls its endpoints together with Hooke's law when it
 * is longer than its rest length and breaks when that force exceeds its
 * limit; nodes that no longer reach an anchor node through springs are
 * removed with a frontier BFS.  One iteration:
 *   (1) pull:     every pull node moves by v dt;
 *   (2) compute:  `substeps` times
 *        (a) per spring: d = p2 - p1, len = sqrt(dx dx + dy dy),
 *            F = k (len - L0) if len > L0 else 0; F > max_force breaks the
 *            spring (it leaves both endpoints' spring arrays; a node whose
 *            spring count drops to zero is deleted), else the spring keeps
 *            the force on p1, f = F (d / len) (p2 receives -f);
 *        (b) per ordinary node: the sum of its springs' forces in slot order
 *            (+f where it is p1, -f where it is p2), a = sum / m,
 *            v = (v + a dt) (1 - damping), x = x + v dt;
 *   (3) remove:   distance 0 at anchor nodes (not pull nodes), infinity
 *            elsewhere; level l visits the neighbours (through its springs)
 *            of every node at distance l and gives the unvisited ones l + 1,
 *            until a level has no node at distance l; a node left at
 *            infinity flags all its springs, and every flagged spring leaves
 *            both endpoints (deleting a node at count zero) and is deleted.
 * Arithmetic is FP32 in the order written above, no contraction (the
 * library is built with -ffp-contract=off).  Deletions within a phase do
 * not interact: a node is deleted only after all its springs are gone, so
 * the result does not depend on the order in which objects are processed.
 *
 * Readings (the thesis gives the steps, not the arithmetic): springs act
 * only when stretched (Hooke's law "beyond its initial length"); the force
 * breaks a spring when strictly above the limit; a node with no spring
 * left is deleted (the thesis' remove_spring); the pull moves once per
 * iteration by v dt; symplectic Euler with a velocity damping factor; a
 * node that never had a spring stays (the BFS removal flags springs only).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define INF_DIST 0x7FFFFFFF

typedef struct {
  int N, S;
  const int8_t* kind;
  float *x, *y, *vx, *vy;
  const float* m;
  int32_t* slot;    /* 3 N spring ids, -1 = empty */
  int32_t* nspr;
  uint8_t* nalive;
  const int32_t *p1, *p2;
  const float *k, *L0, *fmax;
  float *fx, *fy;
  uint8_t* salive;
  int32_t* dist;
} Mesh;

/* a spring leaves one endpoint; the endpoint is deleted at count zero */
static void unlink_end(Mesh* w, int node, int s, int64_t* nodes_deleted) {
  for (int i = 0; i < 3; ++i)
    if (w->slot[3 * node + i] == s) {
      w->slot[3 * node + i] = -1;
      if (--w->nspr[node] == 0) { w->nalive[node] = 0; ++*nodes_deleted; }
      return;
    }
}

static void remove_spring(Mesh* w, int s, int64_t* nodes_deleted) {
  unlink_end(w, w->p1[s], s, nodes_deleted);
  unlink_end(w, w->p2[s], s, nodes_deleted);
  w->salive[s] = 0;
}

static void phase_pull(Mesh* w, float dt) {
  for (int v = 0; v < w->N; ++v)
    if (w->nalive[v] && w->kind[v] == ORC_STRUCT_PULL) {
      w->x[v] = w->x[v] + w->vx[v] * dt;
      w->y[v] = w->y[v] + w->vy[v] * dt;
    }
}

static void phase_forces(Mesh* w, int64_t* broken, int64_t* nodes_deleted) {
  for (int s = 0; s < w->S; ++s) {
    if (!w->salive[s]) continue;
    const int a = w->p1[s], b = w->p2[s];
    const float dx = w->x[b] - w->x[a], dy = w->y[b] - w->y[a];
    const float len = sqrtf(dx * dx + dy * dy);
    const float stretch = len - w->L0[s];
    const float F = stretch > 0.0f ? w->k[s] * stretch : 0.0f;
    if (F > w->fmax[s]) {
      remove_spring(w, s, nodes_deleted);
      ++*broken;
      continue;
    }
    if (F > 0.0f) {
      w->fx[s] = F * (dx / len);
      w->fy[s] = F * (dy / len);
    } else {
      w->fx[s] = 0.0f;
      w->fy[s] = 0.0f;
    }
  }
}

static void phase_move(Mesh* w, float dt, float keep) {
  for (int v = 0; v < w->N; ++v) {
    if (!w->nalive[v] || w->kind[v] != ORC_STRUCT_NODE) continue;
    float Fx = 0.0f, Fy = 0.0f;
    for (int i = 0; i < 3; ++i) {
      const int s = w->slot[3 * v + i];
      if (s < 0) continue;
      if (w->p1[s] == v) { Fx = Fx + w->fx[s]; Fy = Fy + w->fy[s]; }
      else { Fx = Fx - w->fx[s]; Fy = Fy - w->fy[s]; }
    }
    const float ax = Fx / w->m[v], ay = Fy / w->m[v];
    w->vx[v] = (w->vx[v] + ax * dt) * keep;
    w->vy[v] = (w->vy[v] + ay * dt) * keep;
    w->x[v] = w->x[v] + w->vx[v] * dt;
    w->y[v] = w->y[v] + w->vy[v] * dt;
  }
}

/* returns the number of BFS levels run (the last one found no frontier) */
static int64_t phase_remove(Mesh* w, int64_t* springs_deleted, int64_t* nodes_deleted) {
  for (int v = 0; v < w->N; ++v)
    w->dist[v] = (w->nalive[v] && w->kind[v] == ORC_STRUCT_ANCHOR) ? 0 : INF_DIST;
  int64_t levels = 0;
  for (int32_t l = 0;; ++l) {
    ++levels;
    int frontier = 0;
    for (int v = 0; v < w->N; ++v) {
      if (!w->nalive[v] || w->dist[v] != l) continue;
      frontier = 1;
      for (int i = 0; i < 3; ++i) {
        const int s = w->slot[3 * v + i];
        if (s < 0) continue;
        const int u = w->p1[s] == v ? w->p2[s] : w->p1[s];
        if (w->dist[u] == INF_DIST) w->dist[u] = l + 1;
      }
    }
    if (!frontier) break;
  }
  /* flag the springs of unreached nodes, then delete the flagged springs */
  uint8_t* flag = (uint8_t*)calloc((size_t)(w->S > 0 ? w->S : 1), 1);
  for (int v = 0; v < w->N; ++v) {
    if (!w->nalive[v] || w->dist[v] != INF_DIST) continue;
    for (int i = 0; i < 3; ++i)
      if (w->slot[3 * v + i] >= 0) flag[w->slot[3 * v + i]] = 1;
  }
  for (int s = 0; s < w->S; ++s)
    if (w->salive[s] && flag[s]) { remove_spring(w, s, nodes_deleted); ++*springs_deleted; }
  free(flag);
  return levels;
}

int orc_structure_run(int N, int S, const orc_structure_params* p, const int8_t* kind, float* x, float* y,
                      float* vx, float* vy, const float* m, int32_t* slot, int32_t* nspr, uint8_t* nalive,
                      const int32_t* p1, const int32_t* p2, const float* k, const float* L0, const float* fmax,
                      float* fx, float* fy, uint8_t* salive, int32_t* dist, int T, int phases,
                      int64_t* counters) {
  if (N < 1 || S < 0 || !p || !kind || !x || !y || !vx || !vy || !m || !slot || !nspr || !nalive || T < 0 ||
      (S > 0 && (!p1 || !p2 || !k || !L0 || !fmax || !fx || !fy || !salive)) || !dist || p->substeps < 0)
    return -1;
  for (int s = 0; s < S; ++s)
    if (p1[s] < 0 || p1[s] >= N || p2[s] < 0 || p2[s] >= N || p1[s] == p2[s]) return -1;
  Mesh w = {N, S, kind, x, y, vx, vy, m, slot, nspr, nalive, p1, p2, k, L0, fmax, fx, fy, salive, dist};
  const float keep = 1.0f - p->damping;
  for (int t = 0; t < T; ++t) {
    int64_t c[5] = {0, 0, 0, 0, 0};  /* broken, deleted by breaks, BFS springs, BFS nodes, levels */
    if (phases & ORC_STRUCT_PHASE_PULL) phase_pull(&w, p->dt);
    if (phases & ORC_STRUCT_PHASE_COMPUTE)
      for (int sub = 0; sub < p->substeps; ++sub) {
        phase_forces(&w, &c[0], &c[1]);
        phase_move(&w, p->dt, keep);
      }
    if (phases & ORC_STRUCT_PHASE_REMOVE) c[4] = phase_remove(&w, &c[2], &c[3]);
    if (counters) memcpy(counters + 5 * (int64_t)t, c, sizeof(c));
  }
  return 0;
}
