/*
 * Nagel-Schreckenberg traffic with traffic controllers -- oracle (test
 * infrastructure only; never linked into the CUDA library).
 *
 * Extends nasch.c with the controllers of the thesis' "traffic" application
 * (Sec. 7.5, "Intersections and Traffic Lights"): a controller guards the
 * entry of a street o with two or more incoming streets and lets one of
 * them through at a time, by giving every other incoming street a speed
 * limit of zero at the crossing.  Three kinds:
 *   traffic light:       a timer; after `phase_len` steps the green moves on
 *                        to the next incoming street (round robin);
 *   smart traffic light: like a traffic light, but when exactly one incoming
 *                        street has a waiting car and it is red, it turns
 *                        green at once (timer restarted);
 *   yield controller:    the first incoming street (in priority order) with
 *                        a waiting car is green.
 * A car is waiting for o if it is within `lookahead` cells of the end of an
 * incoming street whose route in this step leads to o (the lookahead walks
 * back from the crossing; streets are longer than the lookahead, so it stays
 * on the incoming street).
 *
 * Per step t: (0) controllers update, reading the occupancy at step start;
 * then the cars as in nasch.c, except that (c) follows the thesis' "adjust
 * velocity" code figure with speed limits: along the path, an occupied cell
 * stops the car before it; a cell whose limit is below the car's velocity
 * lowers the velocity to the limit if that still reaches the cell, else the
 * car stops before it.  Every cell's limit is v_max except the first cell of
 * a guarded street, whose limit is 0 for cars from a red incoming street.
 * The claim of nasch.c (lowest cell wins) stays as the last safeguard.
 *
 * Readings: incoming streets of o in increasing street id (also the yield
 * priority); green starts on the first incoming street, timer 0; the yield
 * controller keeps its green when no car waits; a controller of a street
 * with fewer than two incoming streets does nothing.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct { int live, cell, v, route, crossing; } CCar;

static int route_of(const orc_nasch_graph* g, uint64_t seed, uint32_t t, int s) {
  if (g->out_deg[s] <= 0) return -1;
  const int L = g->street_len[s];
  const uint32_t r = orc_draw(seed, ORC_TAG_ROUTE, t, (uint32_t)(g->street_start[s] + L - 1), 0);
  return g->out_street[3 * s + (int)(r % (uint32_t)g->out_deg[s])];
}

int orc_nasch_ctrl_run(const orc_nasch_graph* g, const orc_nasch_ctrl* ctl, uint64_t seed,
                       int8_t* car_v, int16_t* green, int16_t* timer, int t0, int T,
                       int64_t* counters) {
  if (!g || !ctl || !car_v || !green || !timer || g->num_streets < 1 || g->num_cells < 1 ||
      T < 0 || ctl->phase_len < 1 || ctl->lookahead < 0)
    return -1;
  const int S = g->num_streets, C = g->num_cells;
  int* street_of = (int*)malloc(sizeof(int) * (size_t)C);
  for (int s = 0; s < S; ++s)
    for (int i = 0; i < g->street_len[s]; ++i) street_of[g->street_start[s] + i] = s;
  /* incoming lists, increasing street id */
  int* nin = (int*)calloc((size_t)S, sizeof(int));
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < g->out_deg[s]; ++k) ++nin[g->out_street[3 * s + k]];
  int* in_off = (int*)malloc(sizeof(int) * (size_t)(S + 1));
  in_off[0] = 0;
  for (int o = 0; o < S; ++o) in_off[o + 1] = in_off[o] + nin[o];
  int* in_list = (int*)malloc(sizeof(int) * (size_t)(in_off[S] + 1));
  int* fill = (int*)calloc((size_t)S, sizeof(int));
  for (int s = 0; s < S; ++s) /* s increasing: lists come out sorted */
    for (int k = 0; k < g->out_deg[s]; ++k) {
      const int o = g->out_street[3 * s + k];
      in_list[in_off[o] + fill[o]++] = s;
    }
  int* occ = (int*)malloc(sizeof(int) * (size_t)C);
  int* claim = (int*)malloc(sizeof(int) * (size_t)S);
  int* waiting = (int*)malloc(sizeof(int) * (size_t)S); /* per street: route target if waiting, else -1 */
  int* green_street = (int*)malloc(sizeof(int) * (size_t)S);
  CCar* car = NULL;
  int ncar = 0, cap = 0;
  for (int c = 0; c < C; ++c) {
    occ[c] = -1;
    if (car_v[c] >= 0) {
      if (ncar == cap) { cap = cap ? 2 * cap : 1024; car = (CCar*)realloc(car, sizeof(CCar) * (size_t)cap); }
      car[ncar].live = 1; car[ncar].cell = c; car[ncar].v = car_v[c];
      occ[c] = ncar++;
    }
  }
  for (int step = 0; step < T; ++step) {
    const uint32_t t = (uint32_t)(t0 + step + 1);
    int64_t spawned = 0, sunk = 0, moved = 0, lost = 0, switches = 0;
    /* (0) controllers */
    for (int s = 0; s < S; ++s) {
      waiting[s] = -1;
      const int o = route_of(g, seed, t, s);
      if (o < 0) continue;
      const int st = g->street_start[s], L = g->street_len[s];
      for (int k = 0; k < ctl->lookahead && k < L; ++k)
        if (occ[st + L - 1 - k] >= 0) { waiting[s] = o; break; }
    }
    for (int o = 0; o < S; ++o) {
      green_street[o] = -1;
      const int n = nin[o], kind = ctl->ctrl_kind[o];
      if (kind < 0 || n < 2) continue;
      const int* in = in_list + in_off[o];
      int gi = green[o], tm = timer[o];
      const int before = gi;
      if (kind == ORC_CTRL_YIELD) {
        for (int i = 0; i < n; ++i)
          if (waiting[in[i]] == o) { gi = i; break; }
      } else {
        int nw = 0, only = -1;
        for (int i = 0; i < n; ++i)
          if (waiting[in[i]] == o) { ++nw; only = i; }
        if (kind == ORC_CTRL_SMART && nw == 1 && only != gi) {
          gi = only;
          tm = 0;
        } else if (++tm >= ctl->phase_len) {
          gi = (gi + 1) % n;
          tm = 0;
        }
      }
      if (gi != before) ++switches;
      green[o] = (int16_t)gi;
      timer[o] = (int16_t)tm;
      green_street[o] = in[gi];
    }
    /* (a)-(d) per car, against the occupancy at step start */
    const int n0 = ncar;
    for (int s = 0; s < S; ++s) claim[s] = -1;
    for (int i = 0; i < n0; ++i) {
      CCar* a = &car[i];
      if (!a->live) continue;
      const int s = street_of[a->cell], L = g->street_len[s];
      const int p = a->cell - g->street_start[s];
      int v = a->v + 1 < g->v_max ? a->v + 1 : g->v_max;              /* (a) */
      const int o = route_of(g, seed, t, s);                            /* (b) */
      for (int d = 1; d <= v; ++d) {                                    /* (c) */
        const int q = p + d;
        int cell, limit = g->v_max;
        if (q < L) {
          cell = g->street_start[s] + q;
        } else if (o >= 0) {
          cell = g->street_start[o] + (q - L);
          if (q == L && green_street[o] >= 0 && green_street[o] != s) limit = 0;
        } else if (g->sinks_enabled) {
          continue; /* leaving the network: free, no limit */
        } else {
          v = d - 1; /* dead end */
          break;
        }
        if (occ[cell] >= 0) { v = d - 1; break; }
        if (v > limit) {
          if (limit > d - 1) v = limit;
          else { v = d - 1; break; }
        }
      }
      if (v > 0 && orc_draw(seed, ORC_TAG_BRAKE, t, (uint32_t)a->cell, 0) < g->brake_threshold)
        --v;                                                            /* (d) */
      a->v = v;
      a->route = o;
      a->crossing = (o >= 0 && p + v >= L);
      if (a->crossing) {
        const int w = claim[o];
        if (w < 0 || car[w].cell > a->cell) claim[o] = i;
      }
    }
    /* crossing resolution, move, sink */
    for (int i = 0; i < n0; ++i) {
      CCar* a = &car[i];
      if (!a->live) continue;
      const int s = street_of[a->cell], L = g->street_len[s];
      const int p = a->cell - g->street_start[s];
      if (a->crossing && claim[a->route] != i) {
        a->v = L - 1 - p;
        a->crossing = 0;
        ++lost;
      }
      if (g->out_deg[s] == 0 && g->sinks_enabled && p + a->v >= L - 1) {
        occ[a->cell] = -1;
        a->live = 0;
        ++sunk;
        continue;
      }
      if (a->v == 0) continue;
      const int q = p + a->v;
      const int dst = q < L ? g->street_start[s] + q : g->street_start[a->route] + (q - L);
      if (occ[a->cell] == i) occ[a->cell] = -1;
      a->cell = dst;
      ++moved;
    }
    for (int i = 0; i < n0; ++i)
      if (car[i].live) occ[car[i].cell] = i;
    if (g->sources_enabled)
      for (int s = 0; s < S; ++s) {
        if (!g->is_source[s]) continue;
        const int c = g->street_start[s];
        if (occ[c] >= 0) continue;
        if (ncar == cap) { cap = cap ? 2 * cap : 1024; car = (CCar*)realloc(car, sizeof(CCar) * (size_t)cap); }
        car[ncar].live = 1; car[ncar].cell = c; car[ncar].v = 0;
        occ[c] = ncar++;
        ++spawned;
      }
    int w = 0;
    for (int i = 0; i < ncar; ++i)
      if (car[i].live) { car[w] = car[i]; occ[car[w].cell] = w; ++w; }
    ncar = w;
    if (counters) {
      int64_t* k = counters + 6 * (int64_t)step;
      k[0] = ncar; k[1] = spawned; k[2] = sunk; k[3] = moved; k[4] = lost; k[5] = switches;
    }
  }
  for (int c = 0; c < C; ++c) car_v[c] = occ[c] >= 0 ? (int8_t)car[occ[c]].v : (int8_t)-1;
  free(street_of); free(nin); free(in_off); free(in_list); free(fill); free(occ); free(claim);
  free(waiting); free(green_street); free(car);
  return 0;
}
