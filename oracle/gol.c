/*
 * Game of Life with dynamic Alive/Candidate objects -- oracle (test
 * infrastructure only; never linked into the CUDA library).
 *
 * Follows the thesis, Sec. 7.8 ("gol"): classes Cell, abstract Agent,
 * Alive and Candidate; four parallel do-alls per generation:
 *   1. Candidate::prepare  -- decide delete / upgrade / keep,
 *   2. Alive::prepare      -- decide die / stay,
 *   3. Candidate::update   -- perform the candidate action,
 *   4. Alive::update       -- perform the alive action; a newly created Alive
 *      creates Candidates on empty surrounding cells, one creator per cell
 *      chosen by a fixed scan order of the empty cell's neighbourhood
 *      (dx outer, dy inner, both -1..1), as in the "create candidates" code
 *      figure of Sec. 7.8.
 * Readings (where the thesis is silent): torus instead of a bounded grid;
 * a candidate with no alive neighbour is deleted; is_new is cleared in step 2
 * of the following generation; step 4 sees the occupancy left by step 3.
 *
 * The simulation keeps explicit object records (array of structs) and a
 * per-cell occupancy index, exactly as the object model describes; it runs
 * the do-alls one after the other, each over the objects that existed when
 * the do-all started (SMMO semantics, Sec. 5.1.1).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

enum { ACT_KEEP = 0, ACT_BORN = 1, ACT_DELETE = 2, ACT_DIE = 3 };

typedef struct {
  int live;       /* 0 after destroy */
  int kind;       /* ORC_ALIVE or ORC_CANDIDATE */
  int cell;
  uint8_t is_new; /* Alive only */
  uint8_t action;
} Agent;

typedef struct {
  Agent* a;
  int n, cap;
} AgentVec;

static int agent_new(AgentVec* v, int kind, int cell, uint8_t is_new) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 1024;
    v->a = (Agent*)realloc(v->a, (size_t)v->cap * sizeof(Agent));
  }
  Agent* g = &v->a[v->n];
  g->live = 1; g->kind = kind; g->cell = cell; g->is_new = is_new;
  g->action = ACT_KEEP;
  return v->n++;
}

static int wrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* number of Alive objects among the 8 torus neighbours of cell c */
static int alive_neighbours(const AgentVec* v, const int* occ, int W, int H,
                            int c) {
  int x = c % W, y = c / W, n = 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy) {
      if (dx == 0 && dy == 0) continue;
      int o = occ[wrap(y + dy, H) * W + wrap(x + dx, W)];
      if (o >= 0 && v->a[o].kind == ORC_ALIVE) ++n;
    }
  return n;
}

int orc_gol_run(int W, int H, uint8_t* kind, uint8_t* state, int T,
                int64_t* counters) {
  if (W < 3 || H < 3 || !kind || !state || T < 0) return -1;
  const int N = W * H;
  AgentVec v = {0};
  int* occ = (int*)malloc(sizeof(int) * (size_t)N);
  int* occ3 = (int*)malloc(sizeof(int) * (size_t)N);
  int* creator = (int*)malloc(sizeof(int) * (size_t)N);
  for (int c = 0; c < N; ++c) {
    occ[c] = -1;
    if (kind[c] == ORC_ALIVE) occ[c] = agent_new(&v, ORC_ALIVE, c, state[c]);
    else if (kind[c] == ORC_CANDIDATE) occ[c] = agent_new(&v, ORC_CANDIDATE, c, 0);
  }
  for (int t = 0; t < T; ++t) {
    int64_t births = 0, deaths = 0, created = 0, deleted = 0;
    const int n_start = v.n; /* objects existing at generation start */
    /* Step 1: Candidate::prepare */
    for (int i = 0; i < n_start; ++i) {
      Agent* g = &v.a[i];
      if (!g->live || g->kind != ORC_CANDIDATE) continue;
      int n = alive_neighbours(&v, occ, W, H, g->cell);
      g->action = n == 3 ? ACT_BORN : (n == 0 ? ACT_DELETE : ACT_KEEP);
    }
    /* Step 2: Alive::prepare */
    for (int i = 0; i < n_start; ++i) {
      Agent* g = &v.a[i];
      if (!g->live || g->kind != ORC_ALIVE) continue;
      g->is_new = 0;
      int n = alive_neighbours(&v, occ, W, H, g->cell);
      g->action = (n == 2 || n == 3) ? ACT_KEEP : ACT_DIE;
    }
    /* Step 3: Candidate::update (over candidates existing now) */
    const int n3 = v.n;
    for (int i = 0; i < n3; ++i) {
      Agent* g = &v.a[i];
      if (!g->live || g->kind != ORC_CANDIDATE) continue;
      if (g->action == ACT_BORN) {
        int c = g->cell;
        g->live = 0;                              /* destroy(this) */
        occ[c] = agent_new(&v, ORC_ALIVE, c, 1);  /* new Alive(is_new) */
        ++births;
      } else if (g->action == ACT_DELETE) {
        occ[g->cell] = -1;
        v.a[i].live = 0;
        ++deleted;
      }
    }
    /* Step 4: Alive::update over Alive objects existing after step 3.
     * Creation decisions read the occupancy left by step 3. */
    memcpy(occ3, occ, sizeof(int) * (size_t)N);
    const int n4 = v.n;
    for (int c = 0; c < N; ++c) creator[c] = -1;
    for (int i = 0; i < n4; ++i) {
      Agent* g = &v.a[i];
      if (!g->live || g->kind != ORC_ALIVE || !g->is_new) continue;
      int x = g->cell % W, y = g->cell / W;
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
          int ex = wrap(x + dx, W), ey = wrap(y + dy, H), e = ey * W + ex;
          if (occ3[e] != -1) continue;
          /* responsibility scan over the neighbourhood of the empty cell */
          int first = -1;
          for (int ddx = -1; ddx <= 1 && first < 0; ++ddx)
            for (int ddy = -1; ddy <= 1; ++ddy) {
              int o = occ3[wrap(ey + ddy, H) * W + wrap(ex + ddx, W)];
              if (o >= 0 && v.a[o].kind == ORC_ALIVE && v.a[o].is_new) {
                first = o;
                break;
              }
            }
          if (first == i) creator[e] = i;
        }
    }
    for (int i = 0; i < n4; ++i) {
      Agent* g = &v.a[i];
      if (!g->live || g->kind != ORC_ALIVE || g->is_new) continue;
      if (g->action == ACT_DIE) {
        int c = g->cell;
        g->live = 0;
        occ[c] = agent_new(&v, ORC_CANDIDATE, c, 0);
        ++deaths;
      }
    }
    for (int e = 0; e < N; ++e)
      if (creator[e] >= 0) {
        occ[e] = agent_new(&v, ORC_CANDIDATE, e, 0);
        ++created;
      }
    /* drop dead records so the vector does not grow without bound */
    int w = 0;
    for (int i = 0; i < v.n; ++i)
      if (v.a[i].live) {
        v.a[w] = v.a[i];
        occ[v.a[w].cell] = w;
        ++w;
      }
    v.n = w;
    if (counters) {
      int64_t na = 0, nc = 0;
      for (int i = 0; i < v.n; ++i) { if (v.a[i].kind == ORC_ALIVE) ++na; else ++nc; }
      int64_t* k = counters + 7 * (int64_t)t;
      k[0] = na; k[1] = nc; k[2] = births; k[3] = deaths; k[4] = created;
      k[5] = deleted;
      k[6] = 2 * births + 2 * deaths + created + deleted;
    }
  }
  for (int c = 0; c < N; ++c) {
    kind[c] = ORC_EMPTY; state[c] = 0;
    if (occ[c] >= 0) {
      kind[c] = (uint8_t)v.a[occ[c]].kind;
      state[c] = v.a[occ[c]].kind == ORC_ALIVE ? v.a[occ[c]].is_new : 0;
    }
  }
  free(v.a); free(occ); free(occ3); free(creator);
  return 0;
}
