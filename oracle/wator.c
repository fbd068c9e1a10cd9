/*
 * Wa-Tor predator-prey -- oracle (test infrastructure only).
 *
 * Follows the thesis, Sec. 7.6 ("wa-tor"): classes Cell, abstract Agent,
 * Fish and Shark; one iteration is a fish phase (Cell::prepare,
 * Fish::prepare, Cell::decide, Fish::update) followed by a shark phase with
 * the same four steps.  Agents request one neighbouring cell (fish: an
 * empty one; sharks: a fish cell if any, else an empty one), a cell grants
 * at most one request, granted agents move and leave offspring at their old
 * cell once old enough; sharks eat the fish they move onto and starve when
 * their energy runs out.
 *
 * Readings (where the thesis is silent or random): the grant goes to the
 * requester on the lowest cell index (not a random pick); the target among
 * k candidates is draw % k with draw = Philox(seed; step, cell, tag, inst);
 * breeding happens when age >= breed (age reset to 0), only for agents that
 * moved; sharks lose one energy unit per step, starve at 0 (staying in place
 * and freed in update) and are reset to `starve` on eating; newborns start
 * with age 0 (sharks with energy `starve`).  Directions: 0 = (0,-1),
 * 1 = (+1,0), 2 = (0,+1), 3 = (-1,0).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct {
  int live, kind, cell, target; /* target = cell means "stay" */
  int16_t age, energy;
  uint8_t dying;
} Agent;

typedef struct { Agent* a; int n, cap; } AgentVec;

static int agent_new(AgentVec* v, int kind, int cell, int16_t age,
                     int16_t energy) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 1024;
    v->a = (Agent*)realloc(v->a, (size_t)v->cap * sizeof(Agent));
  }
  Agent* g = &v->a[v->n];
  memset(g, 0, sizeof(*g));
  g->live = 1; g->kind = kind; g->cell = cell; g->target = cell;
  g->age = age; g->energy = energy;
  return v->n++;
}

static int neighbour(int c, int d, int W, int H) {
  int x = c % W, y = c / W;
  static const int DX[4] = {0, 1, 0, -1}, DY[4] = {-1, 0, 1, 0};
  x = (x + DX[d] + W) % W;
  y = (y + DY[d] + H) % H;
  return y * W + x;
}

/* one phase (fish or shark) of step t */
static void phase(int kind, int W, int H, uint64_t seed, uint32_t inst,
                  const orc_wator_params* p, uint32_t t, AgentVec* v, int* occ,
                  int* winner, int64_t* k) {
  const int N = W * H;
  const int n0 = v->n; /* agents existing at phase start */
  /* Cell::prepare: clear all requests */
  for (int c = 0; c < N; ++c) winner[c] = -1;
  /* Agent::prepare */
  for (int i = 0; i < n0; ++i) {
    Agent* g = &v->a[i];
    if (!g->live || g->kind != kind) continue;
    g->age = (int16_t)(g->age + 1);
    g->target = g->cell;
    g->dying = 0;
    if (kind == ORC_SHARK) {
      g->energy = (int16_t)(g->energy - 1);
      if (g->energy == 0) { g->dying = 1; continue; }
    }
    int cand[4], nc = 0;
    if (kind == ORC_SHARK)
      for (int d = 0; d < 4; ++d) {
        int o = occ[neighbour(g->cell, d, W, H)];
        if (o >= 0 && v->a[o].kind == ORC_FISH) cand[nc++] = d;
      }
    if (nc == 0)
      for (int d = 0; d < 4; ++d)
        if (occ[neighbour(g->cell, d, W, H)] < 0) cand[nc++] = d;
    if (nc == 0) continue; /* stay */
    uint32_t r = orc_draw(seed, kind == ORC_FISH ? ORC_TAG_FISH : ORC_TAG_SHARK,
                          t, (uint32_t)g->cell, inst);
    g->target = neighbour(g->cell, cand[r % (uint32_t)nc], W, H);
  }
  /* Cell::decide: the requester on the lowest cell index wins */
  for (int i = 0; i < n0; ++i) {
    Agent* g = &v->a[i];
    if (!g->live || g->kind != kind || g->target == g->cell) continue;
    int w = winner[g->target];
    if (w < 0 || v->a[w].cell > g->cell) winner[g->target] = i;
  }
  /* Agent::update */
  const int breed = kind == ORC_FISH ? p->fish_breed : p->shark_breed;
  for (int i = 0; i < n0; ++i) {
    if (!v->a[i].live || v->a[i].kind != kind) continue;
    if (kind == ORC_SHARK && v->a[i].dying) {
      occ[v->a[i].cell] = -1;
      v->a[i].live = 0;
      ++k[5];
      continue;
    }
    if (v->a[i].target == v->a[i].cell || winner[v->a[i].target] != i) continue;
    const int old = v->a[i].cell, dst = v->a[i].target;
    if (kind == ORC_SHARK && occ[dst] >= 0) {
      /* eat the fish on the target cell (a delete of another class) */
      v->a[occ[dst]].live = 0;
      v->a[i].energy = (int16_t)p->starve;
      ++k[3];
    }
    v->a[i].cell = dst;
    occ[dst] = i;
    ++k[kind == ORC_FISH ? 6 : 7];
    const int ripe = p->breed_strict ? v->a[i].age > breed : v->a[i].age >= breed;
    if (ripe) {
      v->a[i].age = 0;
      int nb = agent_new(v, kind, old, 0,
                         (int16_t)(kind == ORC_SHARK ? p->starve : 0));
      occ[old] = nb;
      ++k[kind == ORC_FISH ? 2 : 4];
    } else {
      occ[old] = -1;
    }
  }
}

int orc_wator_run(int W, int H, uint64_t seed, uint32_t inst,
                  const orc_wator_params* p, int8_t* kind, int16_t* age,
                  int16_t* energy, int t0, int T, int64_t* counters) {
  if (W < 1 || H < 1 || !p || !kind || !age || !energy || T < 0) return -1;
  const int N = W * H;
  AgentVec v = {0};
  int* occ = (int*)malloc(sizeof(int) * (size_t)N);
  int* winner = (int*)malloc(sizeof(int) * (size_t)N);
  for (int c = 0; c < N; ++c) {
    occ[c] = -1;
    if (kind[c] == ORC_FISH || kind[c] == ORC_SHARK)
      occ[c] = agent_new(&v, kind[c], c, age[c], energy[c]);
  }
  for (int s = 0; s < T; ++s) {
    const uint32_t t = (uint32_t)(t0 + s + 1);
    int64_t k[8] = {0};
    phase(ORC_FISH, W, H, seed, inst, p, t, &v, occ, winner, k);
    phase(ORC_SHARK, W, H, seed, inst, p, t, &v, occ, winner, k);
    int w = 0;
    for (int i = 0; i < v.n; ++i)
      if (v.a[i].live) {
        v.a[w] = v.a[i];
        occ[v.a[w].cell] = w;
        ++w;
      }
    v.n = w;
    for (int i = 0; i < v.n; ++i) ++k[v.a[i].kind == ORC_FISH ? 0 : 1];
    if (counters) memcpy(counters + 8 * (int64_t)s, k, sizeof(k));
  }
  for (int c = 0; c < N; ++c) {
    kind[c] = 0; age[c] = 0; energy[c] = 0;
    if (occ[c] >= 0) {
      kind[c] = (int8_t)v.a[occ[c]].kind;
      age[c] = v.a[occ[c]].age;
      energy[c] = v.a[occ[c]].kind == ORC_SHARK ? v.a[occ[c]].energy : 0;
    }
  }
  free(v.a); free(occ); free(winner);
  return 0;
}
