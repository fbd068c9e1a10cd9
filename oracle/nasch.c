/*
 * Nagel-Schreckenberg traffic on a street graph -- oracle (test
 * infrastructure only).
 *
 * Follows the thesis, Sec. 7.5 ("traffic"): streets are split into cells
 * holding at most one Car; each iteration a car (a) accelerates by one up to
 * v_max, (b) computes its path of the next v cells (choosing an outgoing
 * street at an intersection), (c) reduces v to the number of free cells on
 * that path (occupancy at the start of the step; the collision part of the
 * "adjust velocity" code figure, without speed limits), (d) brakes by one
 * with probability p and (e) moves.  Producer streets create cars at their
 * first cell when it is empty; sink streets remove cars that reach their
 * end.
 *
 * Readings (the thesis leaves these to traffic controllers and a biased
 * random walk): the outgoing street at the end of street s in step t is
 * out[s][draw(ROUTE, t, last cell of s) % out_deg(s)]; when several cars
 * would enter the same street in one step the car on the lowest cell index
 * wins and the others stop on the last cell of their own street; a car on a
 * sink street that ends on or passes its last cell is removed; producers
 * spawn with probability 1.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct { int live, cell, v, route, crossing; } Car;

int orc_nasch_run(const orc_nasch_graph* g, uint64_t seed, int8_t* car_v,
                  int t0, int T, int64_t* counters) {
  if (!g || !car_v || g->num_streets < 1 || g->num_cells < 1 || T < 0) return -1;
  const int S = g->num_streets, C = g->num_cells;
  int* street_of = (int*)malloc(sizeof(int) * (size_t)C);
  for (int s = 0; s < S; ++s)
    for (int i = 0; i < g->street_len[s]; ++i) street_of[g->street_start[s] + i] = s;
  int* occ = (int*)malloc(sizeof(int) * (size_t)C);
  int* claim = (int*)malloc(sizeof(int) * (size_t)S); /* winning car per street */
  Car* car = NULL;
  int ncar = 0, cap = 0;
  for (int c = 0; c < C; ++c) {
    occ[c] = -1;
    if (car_v[c] >= 0) {
      if (ncar == cap) { cap = cap ? 2 * cap : 1024; car = (Car*)realloc(car, sizeof(Car) * (size_t)cap); }
      car[ncar].live = 1; car[ncar].cell = c; car[ncar].v = car_v[c];
      occ[c] = ncar++;
    }
  }
  for (int step = 0; step < T; ++step) {
    const uint32_t t = (uint32_t)(t0 + step + 1);
    int64_t spawned = 0, sunk = 0, moved = 0;
    const int n0 = ncar;
    for (int s = 0; s < S; ++s) claim[s] = -1;
    /* (a)-(d) per car, against the occupancy at step start */
    for (int i = 0; i < n0; ++i) {
      Car* a = &car[i];
      if (!a->live) continue;
      const int s = street_of[a->cell], L = g->street_len[s];
      const int p = a->cell - g->street_start[s];
      int v = a->v + 1 < g->v_max ? a->v + 1 : g->v_max;            /* (a) */
      int o = -1;                                                     /* (b) */
      if (g->out_deg[s] > 0) {
        uint32_t r = orc_draw(seed, ORC_TAG_ROUTE, t,
                              (uint32_t)(g->street_start[s] + L - 1), 0);
        o = g->out_street[3 * s + (int)(r % (uint32_t)g->out_deg[s])];
      }
      int free_run = 0;                                               /* (c) */
      for (int k = 1; k <= v; ++k) {
        int q = p + k, cell;
        if (q < L) cell = g->street_start[s] + q;
        else if (o >= 0) cell = g->street_start[o] + (q - L);
        else if (g->sinks_enabled) { free_run = k; continue; } /* exit: free */
        else break;                                             /* dead end */
        if (occ[cell] >= 0) break;
        free_run = k;
      }
      v = free_run;
      if (v > 0 && orc_draw(seed, ORC_TAG_BRAKE, t, (uint32_t)a->cell, 0) <
                       g->brake_threshold)
        --v;                                                          /* (d) */
      a->v = v;
      a->route = o;
      a->crossing = (o >= 0 && p + v >= L);
      if (a->crossing) {
        int w = claim[o];
        if (w < 0 || car[w].cell > a->cell) claim[o] = i;
      }
    }
    /* crossing resolution, move, sink */
    for (int i = 0; i < n0; ++i) {
      Car* a = &car[i];
      if (!a->live) continue;
      const int s = street_of[a->cell], L = g->street_len[s];
      const int p = a->cell - g->street_start[s];
      if (a->crossing && claim[a->route] != i) {
        a->v = L - 1 - p; /* lost the claim: stop at the end of own street */
        a->crossing = 0;
      }
      if (g->out_deg[s] == 0 && g->sinks_enabled && p + a->v >= L - 1) {
        occ[a->cell] = -1;
        a->live = 0;
        ++sunk;
        continue;
      }
      if (a->v == 0) continue;
      int q = p + a->v;
      int dst = q < L ? g->street_start[s] + q : g->street_start[a->route] + (q - L);
      if (occ[a->cell] == i) occ[a->cell] = -1;
      a->cell = dst;
      ++moved;
    }
    for (int i = 0; i < n0; ++i)
      if (car[i].live) occ[car[i].cell] = i;
    /* producers */
    if (g->sources_enabled)
      for (int s = 0; s < S; ++s) {
        if (!g->is_source[s]) continue;
        int c = g->street_start[s];
        if (occ[c] >= 0) continue;
        if (ncar == cap) { cap = cap ? 2 * cap : 1024; car = (Car*)realloc(car, sizeof(Car) * (size_t)cap); }
        car[ncar].live = 1; car[ncar].cell = c; car[ncar].v = 0;
        occ[c] = ncar++;
        ++spawned;
      }
    /* compact records */
    int w = 0;
    for (int i = 0; i < ncar; ++i)
      if (car[i].live) { car[w] = car[i]; occ[car[w].cell] = w; ++w; }
    ncar = w;
    if (counters) {
      int64_t* k = counters + 4 * (int64_t)step;
      k[0] = ncar; k[1] = spawned; k[2] = sunk; k[3] = moved;
    }
  }
  for (int c = 0; c < C; ++c) car_v[c] = occ[c] >= 0 ? (int8_t)car[occ[c]].v : (int8_t)-1;
  free(street_of); free(occ); free(claim); free(car);
  return 0;
}
