/*
 * Generational cellular automaton with dynamic objects ("generation") --
 * oracle (test infrastructure only; never linked into the CUDA library).
 *
 * Follows the thesis' "generation" application (Sec. 7.8, its subsection
 * "generation"): an extension of
 * the object-based Life of Sec. 7.8 (see gol.c) in which an Alive object
 * that dies is not replaced at once: it stays on its cell, blocking it, for
 * a fixed number of generations and only then is replaced by a Candidate,
 * which may later become alive again.  The rule is given as masks over the
 * number n of alive (not dying) Alive objects among the 8 torus neighbours:
 * an alive object survives iff bit n of `survive` is set, a Candidate turns
 * into a new Alive iff bit n of `born` is set; `block` is the number of
 * generations a dead Alive blocks its cell.  The thesis' Burst rule
 * (0235678/3468/255) is survive = {0,2,3,5,6,7,8}, born = {3,4,6,8},
 * block = 255 (the thesis says the cell stays blocked for 255 more
 * iterations); block = 0 with survive {2,3}, born {3} is Life.
 *
 * Per generation, four do-alls over the objects existing when each starts:
 *   1. Candidate::prepare -- born if n in `born`, deleted if n == 0;
 *   2. Alive::prepare     -- clears is_new; an alive object dies if n is not
 *      in `survive`; a blocking one expires once it has blocked `block`
 *      generations, else ages by one;
 *   3. Candidate::update  -- performs the candidate action;
 *   4. Alive::update      -- new Alive objects create Candidates on empty
 *      surrounding cells (creator of an empty cell: the first new Alive of
 *      its neighbourhood in the scan order dx outer, dy inner); a dying
 *      object starts blocking (or, with block == 0, is replaced by a
 *      Candidate); an ageing one ages; an expiring one is replaced by a
 *      Candidate.
 * Readings as in gol.c (torus; a candidate without alive neighbour is
 * deleted; step 4 reads the occupancy left by step 3).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

enum { A_KEEP = 0, A_BORN = 1, A_DELETE = 2, A_DIE = 3, A_AGE = 4, A_EXPIRE = 5 };

typedef struct {
  int live;
  int kind;        /* ORC_ALIVE or ORC_CANDIDATE */
  int cell;
  uint8_t is_new;  /* Alive only */
  uint8_t action;
  uint16_t blocked; /* Alive only: 0 alive, k > 0 dead and blocking for k generations */
} GAgent;

typedef struct {
  GAgent* a;
  int n, cap;
} GVec;

static int gnew(GVec* v, int kind, int cell, uint8_t is_new, uint16_t blocked) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 1024;
    v->a = (GAgent*)realloc(v->a, (size_t)v->cap * sizeof(GAgent));
  }
  GAgent* g = &v->a[v->n];
  g->live = 1; g->kind = kind; g->cell = cell; g->is_new = is_new;
  g->action = A_KEEP; g->blocked = blocked;
  return v->n++;
}

static int gwrap(int a, int n) { a %= n; return a < 0 ? a + n : a; }

/* alive (not blocking) Alive objects among the 8 torus neighbours of c */
static int galive(const GVec* v, const int* occ, int W, int H, int c) {
  int x = c % W, y = c / W, n = 0;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy) {
      if (dx == 0 && dy == 0) continue;
      int o = occ[gwrap(y + dy, H) * W + gwrap(x + dx, W)];
      if (o >= 0 && v->a[o].kind == ORC_ALIVE && v->a[o].blocked == 0) ++n;
    }
  return n;
}

int orc_gen_run(int W, int H, uint32_t survive, uint32_t born, int block,
                uint8_t* kind, uint8_t* state, uint16_t* blocked, int T,
                int64_t* counters) {
  if (W < 3 || H < 3 || !kind || !state || !blocked || T < 0 || block < 0 ||
      block > 65535)
    return -1;
  const int N = W * H;
  GVec v = {0};
  int* occ = (int*)malloc(sizeof(int) * (size_t)N);
  int* occ3 = (int*)malloc(sizeof(int) * (size_t)N);
  int* creator = (int*)malloc(sizeof(int) * (size_t)N);
  for (int c = 0; c < N; ++c) {
    occ[c] = -1;
    if (kind[c] == ORC_ALIVE) occ[c] = gnew(&v, ORC_ALIVE, c, state[c], blocked[c]);
    else if (kind[c] == ORC_CANDIDATE) occ[c] = gnew(&v, ORC_CANDIDATE, c, 0, 0);
  }
  for (int t = 0; t < T; ++t) {
    int64_t births = 0, deaths = 0, expired = 0, created = 0, deleted = 0;
    const int n_start = v.n;
    /* 1. Candidate::prepare */
    for (int i = 0; i < n_start; ++i) {
      GAgent* g = &v.a[i];
      if (!g->live || g->kind != ORC_CANDIDATE) continue;
      int n = galive(&v, occ, W, H, g->cell);
      g->action = ((born >> n) & 1) ? A_BORN : (n == 0 ? A_DELETE : A_KEEP);
    }
    /* 2. Alive::prepare */
    for (int i = 0; i < n_start; ++i) {
      GAgent* g = &v.a[i];
      if (!g->live || g->kind != ORC_ALIVE) continue;
      g->is_new = 0;
      if (g->blocked == 0) {
        int n = galive(&v, occ, W, H, g->cell);
        g->action = ((survive >> n) & 1) ? A_KEEP : A_DIE;
      } else {
        g->action = g->blocked >= block ? A_EXPIRE : A_AGE;
      }
    }
    /* 3. Candidate::update */
    const int n3 = v.n;
    for (int i = 0; i < n3; ++i) {
      GAgent* g = &v.a[i];
      if (!g->live || g->kind != ORC_CANDIDATE) continue;
      if (g->action == A_BORN) {
        int c = g->cell;
        g->live = 0;
        occ[c] = gnew(&v, ORC_ALIVE, c, 1, 0);
        ++births;
      } else if (g->action == A_DELETE) {
        occ[g->cell] = -1;
        g->live = 0;
        ++deleted;
      }
    }
    /* 4. Alive::update; creation decisions read the occupancy after step 3 */
    memcpy(occ3, occ, sizeof(int) * (size_t)N);
    const int n4 = v.n;
    for (int c = 0; c < N; ++c) creator[c] = -1;
    for (int i = 0; i < n4; ++i) {
      GAgent* g = &v.a[i];
      if (!g->live || g->kind != ORC_ALIVE || !g->is_new) continue;
      int x = g->cell % W, y = g->cell / W;
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
          int ex = gwrap(x + dx, W), ey = gwrap(y + dy, H), e = ey * W + ex;
          if (occ3[e] != -1) continue;
          int first = -1;
          for (int ddx = -1; ddx <= 1 && first < 0; ++ddx)
            for (int ddy = -1; ddy <= 1; ++ddy) {
              int o = occ3[gwrap(ey + ddy, H) * W + gwrap(ex + ddx, W)];
              if (o >= 0 && v.a[o].kind == ORC_ALIVE && v.a[o].is_new) {
                first = o;
                break;
              }
            }
          if (first == i) creator[e] = i;
        }
    }
    for (int i = 0; i < n4; ++i) {
      GAgent* g = &v.a[i];
      if (!g->live || g->kind != ORC_ALIVE || g->is_new) continue;
      if (g->action == A_DIE && block > 0) {
        g->blocked = 1;
        ++deaths;
      } else if (g->action == A_AGE) {
        g->blocked = (uint16_t)(g->blocked + 1);
      } else if (g->action == A_DIE || g->action == A_EXPIRE) {
        int c = g->cell;
        if (g->action == A_DIE) ++deaths; else ++expired;
        g->live = 0;
        occ[c] = gnew(&v, ORC_CANDIDATE, c, 0, 0);
      }
    }
    for (int e = 0; e < N; ++e)
      if (creator[e] >= 0) {
        occ[e] = gnew(&v, ORC_CANDIDATE, e, 0, 0);
        ++created;
      }
    int w = 0;
    for (int i = 0; i < v.n; ++i)
      if (v.a[i].live) {
        v.a[w] = v.a[i];
        occ[v.a[w].cell] = w;
        ++w;
      }
    v.n = w;
    if (counters) {
      int64_t na = 0, nb = 0, nc = 0;
      for (int i = 0; i < v.n; ++i) {
        if (v.a[i].kind == ORC_CANDIDATE) ++nc;
        else if (v.a[i].blocked) ++nb;
        else ++na;
      }
      int64_t* k = counters + 8 * (int64_t)t;
      k[0] = na; k[1] = nb; k[2] = nc; k[3] = births; k[4] = deaths;
      k[5] = expired; k[6] = created; k[7] = deleted;
    }
  }
  for (int c = 0; c < N; ++c) {
    kind[c] = ORC_EMPTY; state[c] = 0; blocked[c] = 0;
    if (occ[c] >= 0) {
      const GAgent* g = &v.a[occ[c]];
      kind[c] = (uint8_t)g->kind;
      if (g->kind == ORC_ALIVE) { state[c] = g->is_new; blocked[c] = g->blocked; }
    }
  }
  free(v.a); free(occ); free(occ3); free(creator);
  return 0;
}
