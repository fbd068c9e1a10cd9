"""Planted mistakes in the oracle: each pin set must catch them.

Each case copies the oracle (C sources and wrapper) under the oracle's
build folder, plants one plausible mistake in one C file (a flipped sign
or comparison, a dropped term, a swapped index or order, a wrong counter),
checks that the copy still compiles, and runs that oracle's pin module
against it: the case passes when a pin fails (or the planted mistake
crashes or never ends).  Mistakes that cannot change any output are not
listed.  This checks the pins, not the CUDA path, and runs on the CPU only.

Opt-in (``SMMO_ORACLE_MUTATIONS=1``): about a hundred cases, several
minutes in all.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
WORK = os.path.join(ORACLE, "_build", "mutants")

pytestmark = pytest.mark.skipif(not os.environ.get("SMMO_ORACLE_MUTATIONS"),
                                reason="opt-in: set SMMO_ORACLE_MUTATIONS=1")

# (id, pin module under tests/test_oracle_*.py, file, text, replacement)
MUTANTS = [
    ('W1', 'wator', 'wator.c', 'v->a[w].cell > g->cell', 'v->a[w].cell < g->cell'),  # highest index wins
    ('W2', 'wator', 'wator.c', 'v->a[i].energy = (int16_t)p->starve;', ''),  # no energy reset on eating
    ('W3', 'wator', 'wator.c', 'g->age = (int16_t)(g->age + 1);', ''),  # no ageing
    ('W4', 'wator', 'wator.c', 'v->a[i].age = 0;\n      int nb', 'int nb'),  # no age reset on breeding
    ('W5', 'wator', 'wator.c', 'if (o >= 0 && v->a[o].kind == ORC_FISH) cand[nc++] = d;', 'if (0) cand[nc++] = d;'),  # sharks do not hunt
    ('W7', 'wator', 'wator.c', 'if (g->energy == 0)', 'if (g->energy < 0)'),  # starve late
    ('W8', 'wator', 'wator.c', '(int16_t)(kind == ORC_SHARK ? p->starve : 0)', '(int16_t)(kind == ORC_SHARK ? p->starve - 1 : 0)'),  # newborn shark energy
    ('W9', 'wator', 'wator.c', '++k[3];', ''),  # eaten not counted
    ('W11', 'wator', 'wator.c', 'if (v->a[i].target == v->a[i].cell || winner[v->a[i].target] != i) continue;', 'if (v->a[i].target == v->a[i].cell) continue;'),  # losers move
    ('W12', 'wator', 'wator.c', 'p->breed_strict ? v->a[i].age > breed', '!p->breed_strict ? v->a[i].age > breed'),  # breed comparison swapped
    ('W13', 'wator', 'wator.c', '    phase(ORC_FISH, W, H, seed, inst, p, t, &v, occ, winner, k);\n    phase(ORC_SHARK, W, H, seed, inst, p, t, &v, occ, winner, k);', '    phase(ORC_SHARK, W, H, seed, inst, p, t, &v, occ, winner, k);\n    phase(ORC_FISH, W, H, seed, inst, p, t, &v, occ, winner, k);'),  # shark phase first
    ('G1', 'gol', 'gol.c', 'n == 3 ? ACT_BORN', 'n == 2 ? ACT_BORN'),  # born on 2
    ('G2', 'gol', 'gol.c', '(n == 2 || n == 3) ? ACT_KEEP', '(n == 3) ? ACT_KEEP'),  # survive only on 3
    ('G3', 'gol', 'gol.c', 'n == 0 ? ACT_DELETE', 'n <= 1 ? ACT_DELETE'),  # delete candidates with one neighbour
    ('G4', 'gol', 'gol.c', '      if (dx == 0 && dy == 0) continue;\n', ''),  # counts itself
    ('G6', 'gol', 'gol.c', '      g->is_new = 0;\n', ''),  # is_new never cleared
    ('G7', 'gol', 'gol.c', 'return a < 0 ? a + n : a;', 'return a < 0 ? 0 : a;'),  # clamp instead of wrap
    ('G8', 'gol', 'gol.c', 'occ[c] = agent_new(&v, ORC_CANDIDATE, c, 0);\n        ++deaths;', 'occ[c] = -1;\n        ++deaths;'),  # dead cell left empty
    ('G10', 'gol', 'gol.c', 'k[6] = 2 * births + 2 * deaths + created + deleted;', 'k[6] = births + deaths + created + deleted;'),  # alloc op count
    ('N1', 'nasch', 'nasch.c', 'int v = a->v + 1 < g->v_max ? a->v + 1 : g->v_max;', 'int v = g->v_max;'),  # instant acceleration
    ('N2', 'nasch', 'nasch.c', '        --v;                                                          /* (d) */', '        v = v;'),  # no braking
    ('N3', 'nasch', 'nasch.c', 'car[w].cell > a->cell', 'car[w].cell < a->cell'),  # highest cell wins claim
    ('N4', 'nasch', 'nasch.c', 'if (occ[cell] >= 0) break;', 'if (occ[cell] >= 0) { free_run = k; break; }'),  # drives into occupied cell
    ('N5', 'nasch', 'nasch.c', 'a->v = L - 1 - p; /* lost', 'a->v = 0; /* lost'),  # loser stops in place
    ('N6', 'nasch', 'nasch.c', 'p + a->v >= L - 1) {', 'p + a->v >= L) {'),  # sink condition
    ('N7', 'nasch', 'nasch.c', 'if (v > 0 && orc_draw(seed, ORC_TAG_BRAKE', 'if (v > 1 && orc_draw(seed, ORC_TAG_BRAKE'),  # no brake from 1
    ('N8', 'nasch', 'nasch.c', 'if (occ[c] >= 0) continue;\n        if (ncar', 'if (0) continue;\n        if (ncar'),  # spawn over a car
    ('GE1', 'generation', 'generation.c', ' && v->a[o].blocked == 0) ++n;', ') ++n;'),  # blocking cells counted
    ('GE2', 'generation', 'generation.c', 'g->blocked >= block ? A_EXPIRE', 'g->blocked > block ? A_EXPIRE'),  # expire late
    ('GE3', 'generation', 'generation.c', '      g->is_new = 0;\n      if (g->blocked == 0)', '      if (g->blocked == 0)'),  # is_new kept
    ('GE4', 'generation', 'generation.c', '        g->blocked = 1;\n', '        g->blocked = 2;\n'),  # blocking starts at 2
    ('GE5', 'generation', 'generation.c', 'if (g->action == A_DIE) ++deaths; else ++expired;', '++deaths;'),  # expiries counted as deaths
    ('GE6', 'generation', 'generation.c', 'k[0] = na; k[1] = nb;', 'k[0] = na + nb; k[1] = nb;'),  # blocking counted alive
    ('GE7', 'generation', 'generation.c', '((born >> n) & 1) ? A_BORN', '((survive >> n) & 1) ? A_BORN'),  # born uses survive mask
    ('GE8', 'generation', 'generation.c', 'k[6] = created; k[7] = deleted;', 'k[6] = created; k[7] = created;'),  # deleted counter
    ('GE9', 'generation', 'generation.c', '(n == 0 ? A_DELETE : A_KEEP)', '(n <= 1 ? A_DELETE : A_KEEP)'),  # delete with one neighbour
    ('C1', 'nasch_ctrl', 'nasch_ctrl.c', 'k < ctl->lookahead && k < L', 'k <= ctl->lookahead && k < L'),  # lookahead off by one
    ('C2', 'nasch_ctrl', 'nasch_ctrl.c', 'if (waiting[in[i]] == o) { gi = i; break; }', 'if (waiting[in[i]] == o) { gi = i; }'),  # yield picks the last
    ('C3', 'nasch_ctrl', 'nasch_ctrl.c', 'nw == 1 && only != gi', 'nw >= 1 && only != gi'),  # smart with several waiting
    ('C4', 'nasch_ctrl', 'nasch_ctrl.c', 'gi = only;\n          tm = 0;', 'gi = only;'),  # smart timer kept
    ('C5', 'nasch_ctrl', 'nasch_ctrl.c', 'green_street[o] >= 0 && green_street[o] != s) limit = 0;', 'green_street[o] >= 0) limit = 0;'),  # green also limited
    ('C7', 'nasch_ctrl', 'nasch_ctrl.c', 'if (gi != before) ++switches;', '++switches;'),  # switches counted always
    ('C8', 'nasch_ctrl', 'nasch_ctrl.c', '        ++lost;\n', ''),  # lost not counted
    ('C10', 'nasch_ctrl', 'nasch_ctrl.c', 'else if (++tm >= ctl->phase_len)', 'else if (++tm > ctl->phase_len)'),  # phase one step long
    ('C11', 'nasch_ctrl', 'nasch_ctrl.c', 'if (waiting[in[i]] == o) { ++nw; only = i; }', 'if (waiting[in[i]] >= 0) { ++nw; only = i; }'),  # waiting ignores the route
    ('C12', 'nasch_ctrl', 'nasch_ctrl.c', 'if (kind < 0 || n < 2) continue;', 'if (kind < 0 || n < 1) continue;'),  # single-incoming street controlled
    ('C13', 'nasch_ctrl', 'nasch_ctrl.c', 'const int o = route_of(g, seed, t, s);\n      if (o < 0) continue;', 'const int o = route_of(g, seed, t + 1, s);\n      if (o < 0) continue;'),  # controller reads next step route
    ('B1', 'nbody', 'nbody.c', '        float dx = x[j] - x[i];', '        float dx = x[i] - x[j];'),  # force sign x
    ('B2', 'nbody', 'nbody.c', '        float s2 = fmaf(dx, dx, eps2);', '        float s2 = dx * dx;'),  # no softening f32
    ('B3', 'nbody', 'nbody.c', '      z[i] = z[i] + vz[i] * h;\n    }\n    int64_t merges', '    }\n    int64_t merges'),  # z second drift dropped
    ('B4', 'nbody', 'nbody.c', 'return ma < mb || (ma == mb && ia < ib);', 'return ma < mb || (ma == mb && ia > ib);'),  # tie order
    ('B5', 'nbody', 'nbody.c', 'y[t] = (y[j] + y[t]) / 2.0f;', 'y[t] = y[t];'),  # merge y position
    ('B6', 'nbody', 'nbody.c', 'float nvy = (vy[j] * m[j] + vy[t] * m[t]) / nm;', 'float nvy = vy[t];'),  # merge y velocity
    ('B7', 'nbody', 'nbody.c', 'if (pick[b] >= 0 && target[pick[b]] < 0) target[pick[b]] = b;', 'if (pick[b] >= 0) target[pick[b]] = b;'),  # highest receiver
    ('B8', 'nbody', 'nbody.c', 'if (t < 0 || target[t] >= 0) continue;', 'if (t < 0) continue;'),  # chain merge
    ('B10', 'nbody', 'nbody.c', 'u[c] = m[k] * mu[3 * j + c] - m[j] * mu[3 * k + c];', 'u[c] = m[k] * mu[3 * j + c] + m[j] * mu[3 * k + c];'),  # adjoint u sign
    ('B11', 'nbody', 'nbody.c', '    for (size_t k = 0; k < n3; ++k) { lx[k] += g[k]; lv[k] = w[k] + h * lx[k]; }\n  }\n  memcpy(grad, lv', '    for (size_t k = 0; k < n3; ++k) { lx[k] += g[k]; lv[k] = w[k]; }\n  }\n  memcpy(grad, lv'),  # f32traj sweep half kick
    ('B12', 'nbody', 'nbody.c', 'pe -= G * m[i] * m[j] / sqrt(r2);', 'pe -= G * m[i] * m[j] / r2;'),  # potential energy
    ('B13', 'nbody', 'nbody.c', 'P[c] += m[i] * vel[3 * i + c];', 'P[c] += vel[3 * i + c];'),  # momentum mass
    ('B14', 'nbody', 'nbody.c', 's[c] += m[j] * inv * r[c];', 's[c] += m[i] * inv * r[c];'),  # f64 own mass
    ('B15', 'nbody', 'nbody.c', '        float f = m[j] * inv;\n        sx', '        float f = m[i] * inv;\n        sx'),  # f32 own mass
    ('B17', 'nbody', 'nbody.c', 'ax[i] = G * sx; ay[i] = G * sy; az[i] = G * sz;', 'ax[i] = G * sx; ay[i] = G * sy; az[i] = sz;'),  # G on z
    ('B18', 'nbody', 'nbody.c', 'double s2 = r2 + e2, s = sqrt(s2), s3 = s2 * s, s5 = s3 * s2;', 'double s2 = r2, s = sqrt(s2), s3 = s2 * s, s5 = s3 * s2;'),  # adjoint softening
    ('B19', 'nbody', 'nbody.c', '    if (s % ckpt == 0) {', '    if (s % ckpt == 1) {'),  # checkpoint slot
    ('B20', 'nbody', 'nbody.c', '      if (d2 < R2) { pick[b] = j; break; }', '      if (d2 < R2) { pick[b] = j; }'),  # receiver takes last lighter
    ('B21', 'nbody', 'nbody.c', 'x[t] = (x[j] + x[t]) / 2.0f;', 'x[t] = (x[j] * m[j] + x[t] * m[t]) / nm;'),  # centre of mass instead of midpoint
    ('H1', 'barnes_hut', 'barnes_hut.c', 'return (x >= mx ? 1 : 0) + (y >= my ? 2 : 0);', 'return (x > mx ? 1 : 0) + (y >= my ? 2 : 0);'),  # closed lower edge
    ('H2', 'barnes_hut', 'barnes_hut.c', '    sx = sx + cm * cx;', '    sx = sx + cx;'),  # unweighted centre
    ('H3', 'barnes_hut', 'barnes_hut.c', 'if (inside || c->w * c->w >= theta2 * d2)', 'if (c->w * c->w >= theta2 * d2)'),  # no inside rule
    ('H5', 'barnes_hut', 'barnes_hut.c', 'if (*p < 0.0f) { *p = -*p; *v = -*v; }', 'if (*p < 0.0f) { *p = -*p; }'),  # low wall keeps velocity
    ('H6', 'barnes_hut', 'barnes_hut.c', '  if (*p > 0x1.fffffep-1f) *p = 0x1.fffffep-1f;\n', ''),  # no clamp
    ('H7', 'barnes_hut', 'barnes_hut.c', '      vx[b] = vx[b] + (p->G * ax[b]) * p->dt;\n      vy[b] = vy[b] + (p->G * ay[b]) * p->dt;\n      x[b] = x[b] + vx[b] * p->dt;\n', '      x[b] = x[b] + vx[b] * p->dt;\n      vx[b] = vx[b] + (p->G * ax[b]) * p->dt;\n      vy[b] = vy[b] + (p->G * ay[b]) * p->dt;\n'),  # explicit Euler in x
    ('H8', 'barnes_hut', 'barnes_hut.c', 'vx[b] = vx[b] + (p->G * ax[b]) * p->dt;', 'vx[b] = vx[b] + ax[b] * p->dt;'),  # G dropped in x
    ('H9', 'barnes_hut', 'barnes_hut.c', 'counters[2 * (int64_t)t + 1] = visits;', 'counters[2 * (int64_t)t + 1] = visits / 2;'),  # visits counter
    ('H10', 'barnes_hut', 'barnes_hut.c', '  *p1y = q->p1y + ((i & 2) ? h : 0.0f);', '  *p1y = q->p1y + ((i & 1) ? h : 0.0f);'),  # child square y
    ('H11', 'barnes_hut', 'barnes_hut.c', 'const float inv = 1.0f / (s2 * sqrtf(s2));', 'const float inv = 1.0f / s2;'),  # pair power
    ('H12', 'barnes_hut', 'barnes_hut.c', 'if (counters) { counters[2 * (int64_t)t] = tr.count;', 'if (counters) { counters[2 * (int64_t)t] = tr.count - 1;'),  # node counter
    ('F1', 'bfs', 'bfs.c', 'const int v = q[head++];', 'const int v = q[--tail];'),  # stack instead of queue
    ('F2', 'bfs', 'bfs.c', 'if (levels) *levels = maxd + 1;', 'if (levels) *levels = maxd;'),  # level count
    ('S2', 'structure', 'structure.c', 'if (F > w->fmax[s]) {', 'if (F >= w->fmax[s]) {'),  # non-strict break
    ('S3', 'structure', 'structure.c', 'if (--w->nspr[node] == 0) { w->nalive[node] = 0; ++*nodes_deleted; }', '--w->nspr[node];'),  # node never deleted
    ('S4', 'structure', 'structure.c', 'w->fx[s] = F * (dx / len);', 'w->fx[s] = -F * (dx / len);'),  # force sign
    ('S5', 'structure', 'structure.c', 'w->vx[v] = (w->vx[v] + ax * dt) * keep;', 'w->vx[v] = w->vx[v] * keep + ax * dt;'),  # damping placement
    ('S6', 'structure', 'structure.c', '      w->x[v] = w->x[v] + w->vx[v] * dt;\n      w->y[v] = w->y[v] + w->vy[v] * dt;\n    }\n}', '      w->x[v] = w->x[v] + w->vx[v] * dt;\n      w->y[v] = w->y[v] + w->vy[v] * dt * 0.5f;\n    }\n}'),  # half y drift pull
    ('S7', 'structure', 'structure.c', '    w->y[v] = w->y[v] + w->vy[v] * dt;\n  }\n}', '    w->y[v] = w->y[v] + w->vy[v] * dt * 0.5f;\n  }\n}'),  # half y drift node
    ('S8', 'structure', 'structure.c', '(w->nalive[v] && w->kind[v] == ORC_STRUCT_ANCHOR) ? 0 : INF_DIST', '(w->nalive[v] && w->kind[v] != ORC_STRUCT_NODE) ? 0 : INF_DIST'),  # pull nodes as sources
    ('S9', 'structure', 'structure.c', 'if (w->dist[u] == INF_DIST) w->dist[u] = l + 1;', 'if (w->dist[u] == INF_DIST) w->dist[u] = l + 2;'),  # level step
    ('S10', 'structure', 'structure.c', '    if (w->salive[s] && flag[s]) { remove_spring(w, s, nodes_deleted); ++*springs_deleted; }', '    if (w->salive[s] && flag[s]) { w->salive[s] = 0; ++*springs_deleted; }'),  # flagged spring stays linked
    ('S11', 'structure', 'structure.c', 'const float keep = 1.0f - p->damping;', 'const float keep = 1.0f;'),  # no damping
    ('S12', 'structure', 'structure.c', '        phase_forces(&w, &c[0], &c[1]);\n        phase_move(&w, p->dt, keep);\n', '        phase_forces(&w, &c[0], &c[1]);\n        phase_move(&w, p->dt, keep);\n        if (sub) break;\n'),  # substeps capped at 2
    ('S13', 'structure', 'structure.c', 'const float ax = Fx / w->m[v], ay = Fy / w->m[v];', 'const float ax = Fx, ay = Fy / w->m[v];'),  # mass ignored in x
    ('S14', 'structure', 'structure.c', '      if (w->p1[s] == v) { Fx = Fx + w->fx[s]; Fy = Fy + w->fy[s]; }', '      if (w->p1[s] == v) { Fx = Fx + w->fx[s]; Fy = Fy - w->fy[s]; }'),  # y force sign at p1
    ('S15', 'structure', 'structure.c', '    ++levels;\n', ''),  # level counter
    ('S16', 'structure', 'structure.c', '      ++*broken;\n', ''),  # broken counter
    ('S1b', 'structure', 'structure.c', 'const float F = stretch > 0.0f ? w->k[s] * stretch : 0.0f;', 'const float F = w->k[s] * fabsf(stretch);'),  # compression acts (nonzero)
    ('P1', 'philox', 'philox.c', 'for (int r = 0; r < 10; ++r) {', 'for (int r = 0; r < 9; ++r) {'),  # nine rounds
    ('P2', 'philox', 'philox.c', 'k[1] += 0xBB67AE85u;', 'k[1] += 0xBB67AE84u;'),  # key increment
    ('P3', 'philox', 'philox.c', 'uint32_t n1 = lo1;\n', 'uint32_t n1 = lo0;\n'),  # permutation
    ('P4', 'philox', 'philox.c', 'const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};', 'const uint32_t key[2] = {(uint32_t)(seed >> 32), (uint32_t)seed};'),  # key halves swapped in draw
]


def _limits():
    import resource
    resource.setrlimit(resource.RLIMIT_AS, (6 << 30, 6 << 30))


@pytest.mark.parametrize("mid,module,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(mid, module, fname, old, new):
    dest = os.path.join(WORK, mid)
    if os.path.isdir(dest):
        shutil.rmtree(dest)
    shutil.copytree(ORACLE, os.path.join(dest, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__", "_build"))
    path = os.path.join(dest, "oracle", fname)
    src = open(path).read()
    assert src.count(old) == 1, "the planted text must occur exactly once"
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([dest, ROOT]))
    built = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__); oracle.build()"],
                           cwd=dest, env=env, capture_output=True, text=True, timeout=300)
    assert built.returncode == 0, built.stderr[-2000:]
    assert built.stdout.startswith(dest)
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                            os.path.join(ROOT, "tests", "test_oracle_%s.py" % module)],
                           cwd=dest, env=env, capture_output=True, text=True, timeout=300, preexec_fn=_limits)
    except subprocess.TimeoutExpired:
        return  # the planted mistake does not terminate: caught
    finally:
        shutil.rmtree(dest, ignore_errors=True)
    assert r.returncode != 0, "no pin of test_oracle_%s.py fails:\n%s" % (module, r.stdout[-1500:])
    if r.returncode > 0:
        assert "failed" in r.stdout.splitlines()[-1], r.stdout[-1500:]
