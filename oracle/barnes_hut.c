/*
 * Barnes-Hut n-body in 2-D with a quad tree -- oracle (test infrastructure
 * only; never linked into the CUDA library).
 *
 * Follows the thesis' "barnes-hut" application (Sec. 7.3): bodies in the
 * unit square [0,1)^2, a quad tree whose tree nodes split their square into
 * four equal quadrants (index (x >= mid_x) + 2 (y >= mid_y)), a bottom-up
 * summary (total mass and centre of gravity of every tree node), a top-down
 * force traversal in preorder (children 0..3), and a body update.
 *
 * The SMMO program keeps one tree alive and maintains it (remove bodies that
 * left their quadrant, reinsert them, collapse empty and single-body tree
 * nodes); after the collapse the tree is the region quad tree of the
 * current positions: a tree node exists exactly where two or more bodies
 * share its square, a square with one body holds the body itself.  That
 * tree is unique, so the oracle simply builds it from the positions at the
 * start of every step (by inserting the bodies one by one).
 *
 * Arithmetic (FP32, fixed order, no contraction):
 *   summary:  m = sum of the children's masses in child order,
 *             c = (sum in child order of m_i c_i) / m, per coordinate;
 *   opening:  a tree node is opened if the body lies in its square or
 *             w^2 >= theta^2 d^2 (w: square width, d: body-to-centre
 *             distance), else its summary acts as one body;
 *   pair:     s2 = (dx dx + dy dy) + eps^2, inv = 1 / (s2 sqrt(s2)),
 *             a += (m inv) d, with d = other - self; a body skips itself;
 *   update:   v += (G a) dt; x += v dt; a coordinate that leaves [0, 1) is
 *             reflected (x -> -x, or x -> 2 - x) and its velocity negated,
 *             then clamped to [0, 1 - 2^-24].
 * Readings: the thesis gives no opening rule beyond "close to the centre of
 * gravity"; this is the classic width / distance < theta criterion.  The
 * thesis' bodies bounce off the walls of the simulation area; the
 * reflection above is that bounce.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct {
  float p1x, p1y, w;   /* square: [p1x, p1x + w) x [p1y, p1y + w) */
  int child[4];        /* -1 empty, >= 0 tree node, <= -2: body -(child + 2) */
  float m, cx, cy;     /* summary */
} QNode;

typedef struct {
  QNode* n;
  int count, cap;
} QTree;

static int qnew(QTree* t, float p1x, float p1y, float w) {
  if (t->count == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 1024;
    t->n = (QNode*)realloc(t->n, sizeof(QNode) * (size_t)t->cap);
  }
  QNode* q = &t->n[t->count];
  q->p1x = p1x; q->p1y = p1y; q->w = w;
  for (int i = 0; i < 4; ++i) q->child[i] = -1;
  q->m = q->cx = q->cy = 0.0f;
  return t->count++;
}

static int quad(const QNode* q, float x, float y) {
  const float h = q->w * 0.5f;  /* exact: widths are powers of two */
  const float mx = q->p1x + h, my = q->p1y + h;
  return (x >= mx ? 1 : 0) + (y >= my ? 2 : 0);
}

static void child_square(const QNode* q, int i, float* p1x, float* p1y, float* w) {
  const float h = q->w * 0.5f;
  *p1x = q->p1x + ((i & 1) ? h : 0.0f);
  *p1y = q->p1y + ((i & 2) ? h : 0.0f);
  *w = h;
}

/* returns 0, or -1 if two bodies could not be separated (same position) */
static int insert(QTree* t, int b, const float* x, const float* y) {
  int cur = 0;
  for (int depth = 0; depth < 60; ++depth) {
    const int i = quad(&t->n[cur], x[b], y[b]);
    const int ch = t->n[cur].child[i];
    if (ch == -1) { t->n[cur].child[i] = -(b + 2); return 0; }
    if (ch >= 0) { cur = ch; continue; }
    const int other = -(ch + 2);
    float p1x, p1y, w;
    child_square(&t->n[cur], i, &p1x, &p1y, &w);
    const int nn = qnew(t, p1x, p1y, w);
    t->n[nn].child[quad(&t->n[nn], x[other], y[other])] = ch;
    t->n[cur].child[i] = nn;
    cur = nn;
  }
  return -1;
}

static void summarize(QTree* t, int q, const float* x, const float* y, const float* m) {
  float ms = 0.0f, sx = 0.0f, sy = 0.0f;
  for (int i = 0; i < 4; ++i) {
    const int ch = t->n[q].child[i];
    if (ch == -1) continue;
    float cm, cx, cy;
    if (ch >= 0) {
      summarize(t, ch, x, y, m);
      cm = t->n[ch].m; cx = t->n[ch].cx; cy = t->n[ch].cy;
    } else {
      const int b = -(ch + 2);
      cm = m[b]; cx = x[b]; cy = y[b];
    }
    ms = ms + cm;
    sx = sx + cm * cx;
    sy = sy + cm * cy;
  }
  t->n[q].m = ms;
  t->n[q].cx = ms > 0.0f ? sx / ms : 0.0f;
  t->n[q].cy = ms > 0.0f ? sy / ms : 0.0f;
}

static void pair(float xi, float yi, float xj, float yj, float mj, float eps2, float* ax, float* ay) {
  const float dx = xj - xi, dy = yj - yi;
  const float s2 = (dx * dx + dy * dy) + eps2;
  const float inv = 1.0f / (s2 * sqrtf(s2));
  const float f = mj * inv;
  *ax = *ax + f * dx;
  *ay = *ay + f * dy;
}

static void force(const QTree* t, int q, int self, const float* x, const float* y, const float* m,
                  float eps2, float theta2, float* ax, float* ay, int64_t* visits) {
  for (int i = 0; i < 4; ++i) {
    const int ch = t->n[q].child[i];
    if (ch == -1) continue;
    ++*visits;
    if (ch < 0) {
      const int b = -(ch + 2);
      if (b != self) pair(x[self], y[self], x[b], y[b], m[b], eps2, ax, ay);
      continue;
    }
    const QNode* c = &t->n[ch];
    const float xs = x[self], ys = y[self];
    const int inside = xs >= c->p1x && xs < c->p1x + c->w && ys >= c->p1y && ys < c->p1y + c->w;
    const float dx = c->cx - xs, dy = c->cy - ys;
    const float d2 = dx * dx + dy * dy;
    if (inside || c->w * c->w >= theta2 * d2)
      force(t, ch, self, x, y, m, eps2, theta2, ax, ay, visits);
    else
      pair(xs, ys, c->cx, c->cy, c->m, eps2, ax, ay);
  }
}

static void bounce(float* p, float* v) {
  if (*p < 0.0f) { *p = -*p; *v = -*v; }
  else if (*p >= 1.0f) { *p = 2.0f - *p; *v = -*v; }
  if (*p < 0.0f) *p = 0.0f;
  if (*p > 0x1.fffffep-1f) *p = 0x1.fffffep-1f;
}

int orc_bh_build(int N, const float* x, const float* y, int* nodes, int* depth_out) {
  if (N < 1 || !x || !y) return -1;
  QTree t = {0};
  qnew(&t, 0.0f, 0.0f, 1.0f);
  int rc = 0;
  for (int b = 0; b < N && !rc; ++b) rc = insert(&t, b, x, y);
  if (nodes) *nodes = t.count;
  if (depth_out) {
    /* depth of the deepest tree node (root = 0) */
    int* d = (int*)calloc((size_t)t.count, sizeof(int));
    int md = 0;
    for (int q = 0; q < t.count; ++q)
      for (int i = 0; i < 4; ++i)
        if (t.n[q].child[i] >= 0) { d[t.n[q].child[i]] = d[q] + 1; if (d[q] + 1 > md) md = d[q] + 1; }
    *depth_out = md;
    free(d);
  }
  free(t.n);
  return rc;
}

int orc_bh_run(int N, const orc_bh_params* p, float* x, float* y, float* vx, float* vy,
               const float* m, int T, int64_t* counters) {
  if (N < 1 || !p || !x || !y || !vx || !vy || !m || T < 0) return -1;
  const float eps2 = p->eps * p->eps, theta2 = p->theta * p->theta;
  float* ax = (float*)malloc(sizeof(float) * (size_t)N);
  float* ay = (float*)malloc(sizeof(float) * (size_t)N);
  int rc = 0;
  for (int t = 0; t < T && !rc; ++t) {
    QTree tr = {0};
    qnew(&tr, 0.0f, 0.0f, 1.0f);
    for (int b = 0; b < N && !rc; ++b) rc = insert(&tr, b, x, y);
    if (rc) { free(tr.n); break; }
    summarize(&tr, 0, x, y, m);
    int64_t visits = 0;
    for (int b = 0; b < N; ++b) {
      ax[b] = 0.0f; ay[b] = 0.0f;
      force(&tr, 0, b, x, y, m, eps2, theta2, &ax[b], &ay[b], &visits);
    }
    for (int b = 0; b < N; ++b) {
      vx[b] = vx[b] + (p->G * ax[b]) * p->dt;
      vy[b] = vy[b] + (p->G * ay[b]) * p->dt;
      x[b] = x[b] + vx[b] * p->dt;
      y[b] = y[b] + vy[b] * p->dt;
      bounce(&x[b], &vx[b]);
      bounce(&y[b], &vy[b]);
    }
    if (counters) { counters[2 * (int64_t)t] = tr.count; counters[2 * (int64_t)t + 1] = visits; }
    free(tr.n);
  }
  free(ax); free(ay);
  return rc;
}

int orc_bh_accel(int N, float eps, float theta, const float* x, const float* y, const float* m,
                 float* ax, float* ay) {
  if (N < 1 || !x || !y || !m || !ax || !ay) return -1;
  QTree tr = {0};
  qnew(&tr, 0.0f, 0.0f, 1.0f);
  int rc = 0;
  for (int b = 0; b < N && !rc; ++b) rc = insert(&tr, b, x, y);
  if (!rc) {
    summarize(&tr, 0, x, y, m);
    int64_t visits = 0;
    for (int b = 0; b < N; ++b) {
      ax[b] = 0.0f; ay[b] = 0.0f;
      force(&tr, 0, b, x, y, m, eps * eps, theta * theta, &ax[b], &ay[b], &visits);
    }
  }
  free(tr.n);
  return rc;
}
