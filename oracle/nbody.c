/*
 * Direct n-body with collision merge, and its adjoint -- oracle (test
 * infrastructure only).
 *
 * Follows the thesis, Sec. 7.1 ("nbody": every body sums the force of all
 * other bodies with a sequential device_do loop, then a second do-all
 * updates velocity and position) and Sec. 7.2 ("collision": pull-style
 * prepare-merge in which a receiving body scans for a lighter body within
 * the merge threshold and stops at the first one, push-style perform-merge
 * that skips a target which is itself being merged, perfectly inelastic
 * merge with v = (v1 m1 + v2 m2)/(m1 + m2), x = (x1 + x2)/2, m = m1 + m2,
 * then deletion of the merged body).
 *
 * Readings: 3-D Plummer-softened gravity a_i = G sum_j m_j r_ij /
 * (|r_ij|^2 + eps^2)^{3/2} with r_ij = x_j - x_i, summed over j in
 * increasing body id; kick-drift-kick is replaced by drift-kick-drift
 * (x += v dt/2; v += a dt; x += v dt/2) so a merge never leaves a stale
 * acceleration; no wall bounce.  The thesis' merge races are made
 * deterministic: "lighter" means (m, id) lexicographically smaller, a body
 * picked by several receivers goes to the lowest receiver id, and a merge
 * into a body that is itself being merged is skipped (as printed).
 *
 * The FP32 path fixes the evaluation order of every operation, with the
 * fused multiply-adds written out (fmaf, one rounding each) and every other
 * product and sum rounded on its own (compiled with -ffp-contract=off, so
 * the compiler fuses nothing else):
 *   dx = xj - xi (same for y, z);
 *   s2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps*eps)));
 *   inv = 1 / (s2 * sqrt(s2)); f = mj * inv;
 *   a = fmaf(f, d, a) per component, j in increasing id; a = G * a.
 *
 * The adjoint (no-merge variant, loss L = 1/2 sum_i m_i |v_i(T)|^2) is the
 * reverse of one drift-kick-drift step with
 *   w = lambda_v + h lambda_x,  mu = dt w,
 *   g_k = G sum_{j != k} H(x1_j - x1_k) (m_k mu_j - m_j mu_k),
 *   H(r) = I / s^3 - 3 r r^T / s^5,  s^2 = |r|^2 + eps^2,
 *   lambda_x <- lambda_x + g,  lambda_v <- w + h lambda_x,
 * where x1 is the mid-step position; (x, v) are checkpointed every `ckpt`
 * steps and each segment is recomputed forward before it is reversed.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the receiver loops below (n <= 0: the OpenMP default).
 * Returns the number now in use (1 without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---------------------------------------------------------------- FP32 */
int orc_nbody_accel_f32(int N, float G, float eps, const float* x,
                        const float* y, const float* z, const float* m,
                        const uint8_t* live, float* ax, float* ay, float* az) {
  if (N < 0) return -1;
  const float eps2 = eps * eps;
  /* receivers are independent; each sums its j in increasing order, so the
   * result does not depend on the number of threads */
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < N; ++i) {
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    if (live[i]) {
      for (int j = 0; j < N; ++j) {
        if (j == i || !live[j]) continue;
        float dx = x[j] - x[i];
        float dy = y[j] - y[i];
        float dz = z[j] - z[i];
        float s2 = fmaf(dx, dx, eps2);
        s2 = fmaf(dy, dy, s2);
        s2 = fmaf(dz, dz, s2);
        float inv = 1.0f / (s2 * sqrtf(s2));
        float f = m[j] * inv;
        sx = fmaf(f, dx, sx);
        sy = fmaf(f, dy, sy);
        sz = fmaf(f, dz, sz);
      }
    }
    ax[i] = G * sx; ay[i] = G * sy; az[i] = G * sz;
  }
  return 0;
}

/* (m_a, id_a) < (m_b, id_b) lexicographically */
static int lighter(float ma, int ia, float mb, int ib) {
  return ma < mb || (ma == mb && ia < ib);
}

static int64_t merge_pass(int N, float R, float* x, float* y, float* z,
                          float* vx, float* vy, float* vz, float* m,
                          uint8_t* live, int* pick, int* target) {
  const float R2 = R * R;
  for (int i = 0; i < N; ++i) { pick[i] = -1; target[i] = -1; }
  /* prepare merge: receiver b scans bodies in id order, stops at the first
   * lighter body within the threshold (receivers are independent) */
#pragma omp parallel for schedule(dynamic, 64)
  for (int b = 0; b < N; ++b) {
    if (!live[b]) continue;
    for (int j = 0; j < N; ++j) {
      if (j == b || !live[j]) continue;
      if (!lighter(m[j], j, m[b], b)) continue;
      float dx = x[j] - x[b];
      float dy = y[j] - y[b];
      float dz = z[j] - z[b];
      float d2 = dx * dx;
      d2 = d2 + dy * dy;
      d2 = d2 + dz * dz;
      if (d2 < R2) { pick[b] = j; break; }
    }
  }
  /* a picked body goes to the lowest receiver id */
  for (int b = 0; b < N; ++b)
    if (pick[b] >= 0 && target[pick[b]] < 0) target[pick[b]] = b;
  /* perform merge (push from the merged body into its target) */
  int64_t merges = 0;
  for (int j = 0; j < N; ++j) {
    int t = target[j];
    if (t < 0 || target[t] >= 0) continue;
    float nm = m[j] + m[t];
    float nvx = (vx[j] * m[j] + vx[t] * m[t]) / nm;
    float nvy = (vy[j] * m[j] + vy[t] * m[t]) / nm;
    float nvz = (vz[j] * m[j] + vz[t] * m[t]) / nm;
    m[t] = nm;
    vx[t] = nvx; vy[t] = nvy; vz[t] = nvz;
    x[t] = (x[j] + x[t]) / 2.0f;
    y[t] = (y[j] + y[t]) / 2.0f;
    z[t] = (z[j] + z[t]) / 2.0f;
    live[j] = 0;
    ++merges;
  }
  return merges;
}

int orc_nbody_run_f32(int N, const orc_nbody_params_f32* p, float* x, float* y,
                      float* z, float* vx, float* vy, float* vz, float* m,
                      uint8_t* live, int T, int64_t* counters) {
  if (N < 0 || !p || T < 0) return -1;
  float* ax = (float*)malloc(sizeof(float) * (size_t)(3 * N + 3));
  float* ay = ax + N + 1;
  float* az = ay + N + 1;
  int* pick = (int*)malloc(sizeof(int) * (size_t)(2 * N + 2));
  int* target = pick + N + 1;
  const float h = 0.5f * p->dt;
  for (int s = 0; s < T; ++s) {
    for (int i = 0; i < N; ++i) {
      if (!live[i]) continue;
      x[i] = x[i] + vx[i] * h;
      y[i] = y[i] + vy[i] * h;
      z[i] = z[i] + vz[i] * h;
    }
    orc_nbody_accel_f32(N, p->G, p->eps, x, y, z, m, live, ax, ay, az);
    for (int i = 0; i < N; ++i) {
      if (!live[i]) continue;
      vx[i] = vx[i] + ax[i] * p->dt;
      vy[i] = vy[i] + ay[i] * p->dt;
      vz[i] = vz[i] + az[i] * p->dt;
      x[i] = x[i] + vx[i] * h;
      y[i] = y[i] + vy[i] * h;
      z[i] = z[i] + vz[i] * h;
    }
    int64_t merges = 0;
    if (p->merge) merges = merge_pass(N, p->merge_r, x, y, z, vx, vy, vz, m, live, pick, target);
    if (counters) counters[s] = merges;
  }
  free(ax); free(pick);
  return 0;
}

/* One no-merge FP32 step evaluated only for the listed receivers (same
 * order of operations as orc_nbody_run_f32): out = 6 floats per listed
 * body (x, y, z, vx, vy, vz after the step). */
int orc_nbody_step_sample_f32(int N, float G, float eps, float dt, const float* x,
                              const float* y, const float* z, const float* vx,
                              const float* vy, const float* vz, const float* m,
                              const uint8_t* live, const int32_t* idx, int nidx,
                              float* out) {
  if (N < 0 || nidx < 0) return -1;
  const float h = 0.5f * dt, eps2 = eps * eps;
  float* x1 = (float*)malloc(sizeof(float) * (size_t)(3 * N + 3));
  float* y1 = x1 + N + 1;
  float* z1 = y1 + N + 1;
  for (int j = 0; j < N; ++j) {
    x1[j] = x[j] + vx[j] * h;
    y1[j] = y[j] + vy[j] * h;
    z1[j] = z[j] + vz[j] * h;
  }
  for (int q = 0; q < nidx; ++q) {
    const int i = idx[q];
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;
    for (int j = 0; j < N; ++j) {
      if (j == i || !live[j]) continue;
      float dx = x1[j] - x1[i];
      float dy = y1[j] - y1[i];
      float dz = z1[j] - z1[i];
      float s2 = fmaf(dx, dx, eps2);
      s2 = fmaf(dy, dy, s2);
      s2 = fmaf(dz, dz, s2);
      float inv = 1.0f / (s2 * sqrtf(s2));
      float f = m[j] * inv;
      sx = fmaf(f, dx, sx);
      sy = fmaf(f, dy, sy);
      sz = fmaf(f, dz, sz);
    }
    float ax = G * sx, ay = G * sy, az = G * sz;
    float nvx = vx[i] + ax * dt, nvy = vy[i] + ay * dt, nvz = vz[i] + az * dt;
    out[6 * q + 0] = x1[i] + nvx * h;
    out[6 * q + 1] = y1[i] + nvy * h;
    out[6 * q + 2] = z1[i] + nvz * h;
    out[6 * q + 3] = nvx;
    out[6 * q + 4] = nvy;
    out[6 * q + 5] = nvz;
  }
  free(x1);
  return 0;
}

/* ---------------------------------------------------------------- FP64 */
int orc_nbody_accel_f64(int N, double G, double eps, const double* pos,
                        const double* m, double* acc) {
  if (N < 0) return -1;
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 64)
  for (int i = 0; i < N; ++i) {
    double s[3] = {0, 0, 0};
    for (int j = 0; j < N; ++j) {
      if (j == i) continue;
      double r[3], r2 = e2;
      for (int c = 0; c < 3; ++c) { r[c] = pos[3 * j + c] - pos[3 * i + c]; r2 += r[c] * r[c]; }
      double inv = 1.0 / (r2 * sqrt(r2));
      for (int c = 0; c < 3; ++c) s[c] += m[j] * inv * r[c];
    }
    for (int c = 0; c < 3; ++c) acc[3 * i + c] = G * s[c];
  }
  return 0;
}

static void step_f64(int N, double G, double eps, double dt, double* pos,
                     double* vel, const double* m, double* acc, double* x1_out) {
  const double h = 0.5 * dt;
  for (int k = 0; k < 3 * N; ++k) pos[k] += vel[k] * h;
  if (x1_out) memcpy(x1_out, pos, sizeof(double) * 3 * (size_t)N);
  orc_nbody_accel_f64(N, G, eps, pos, m, acc);
  for (int k = 0; k < 3 * N; ++k) { vel[k] += acc[k] * dt; pos[k] += vel[k] * h; }
}

int orc_nbody_run_f64(int N, double G, double eps, double dt, double* pos,
                      double* vel, const double* m, int T) {
  if (N < 0 || T < 0) return -1;
  double* acc = (double*)malloc(sizeof(double) * 3 * (size_t)(N + 1));
  for (int s = 0; s < T; ++s) step_f64(N, G, eps, dt, pos, vel, m, acc, NULL);
  free(acc);
  return 0;
}

int orc_nbody_energy_f64(int N, double G, double eps, const double* pos,
                         const double* vel, const double* m, double* E,
                         double* P3) {
  double ke = 0, pe = 0, P[3] = {0, 0, 0};
  for (int i = 0; i < N; ++i) {
    double v2 = 0;
    for (int c = 0; c < 3; ++c) { v2 += vel[3 * i + c] * vel[3 * i + c]; P[c] += m[i] * vel[3 * i + c]; }
    ke += 0.5 * m[i] * v2;
    for (int j = i + 1; j < N; ++j) {
      double r2 = eps * eps;
      for (int c = 0; c < 3; ++c) { double d = pos[3 * j + c] - pos[3 * i + c]; r2 += d * d; }
      pe -= G * m[i] * m[j] / sqrt(r2);
    }
  }
  if (E) *E = ke + pe;
  if (P3) { P3[0] = P[0]; P3[1] = P[1]; P3[2] = P[2]; }
  return 0;
}

int orc_nbody_pair_adjoint_f64(int N, double G, double eps, const double* pos,
                               const double* m, const double* mu, double* g) {
  if (N < 0) return -1;
  const double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 64)
  for (int k = 0; k < N; ++k) {
    double acc[3] = {0, 0, 0};
    for (int j = 0; j < N; ++j) {
      if (j == k) continue;
      double r[3], u[3], r2 = 0;
      for (int c = 0; c < 3; ++c) {
        r[c] = pos[3 * j + c] - pos[3 * k + c];
        r2 += r[c] * r[c];
        u[c] = m[k] * mu[3 * j + c] - m[j] * mu[3 * k + c];
      }
      double s2 = r2 + e2, s = sqrt(s2), s3 = s2 * s, s5 = s3 * s2;
      double ru = r[0] * u[0] + r[1] * u[1] + r[2] * u[2];
      for (int c = 0; c < 3; ++c) acc[c] += u[c] / s3 - 3.0 * r[c] * ru / s5;
    }
    for (int c = 0; c < 3; ++c) g[3 * k + c] = G * acc[c];
  }
  return 0;
}

/* Reverse sweep shared by both adjoints: from lambda_x = 0, lambda_v = m v_T,
 * step s = T-1 .. 0 with the mid-step positions x1[s] (N x 3 each). */
static void reverse_sweep(int N, double G, double eps, double dt, const double* m,
                          const double* x1, int T, const double* vT, double* grad) {
  const size_t n3 = 3 * (size_t)N;
  const double h = 0.5 * dt;
  double* lx = (double*)calloc(n3, sizeof(double));
  double* lv = (double*)malloc(sizeof(double) * n3);
  double* w = (double*)malloc(sizeof(double) * n3);
  double* mu = (double*)malloc(sizeof(double) * n3);
  double* g = (double*)malloc(sizeof(double) * n3);
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) lv[3 * i + c] = m[i] * vT[3 * i + c];
  for (int s = T - 1; s >= 0; --s) {
    for (size_t k = 0; k < n3; ++k) { w[k] = lv[k] + h * lx[k]; mu[k] = dt * w[k]; }
    orc_nbody_pair_adjoint_f64(N, G, eps, x1 + n3 * (size_t)s, m, mu, g);
    for (size_t k = 0; k < n3; ++k) { lx[k] += g[k]; lv[k] = w[k] + h * lx[k]; }
  }
  memcpy(grad, lv, sizeof(double) * n3);
  free(lx); free(lv); free(w); free(mu); free(g);
}

/* FP64 reverse sweep along the FP32 trajectory: the forward pass is the
 * FP32 no-merge step of orc_nbody_run_f32 (same operations), its mid-step
 * positions and final velocities are widened to double, and the reverse
 * sweep runs in FP64.  Isolates the accuracy of an FP32 reverse sweep from
 * the divergence of FP32 and FP64 forward trajectories. */
int orc_nbody_adjoint_f32traj(int N, float G, float eps, float dt, const float* x0,
                              const float* y0, const float* z0, const float* vx0,
                              const float* vy0, const float* vz0, const float* m32,
                              int T, double* grad, double* loss) {
  if (N < 1 || T < 0) return -1;
  const size_t n3 = 3 * (size_t)N;
  float* st = (float*)malloc(sizeof(float) * 6 * (size_t)N);
  float *x = st, *y = st + N, *z = st + 2 * N, *vx = st + 3 * N, *vy = st + 4 * N, *vz = st + 5 * N;
  memcpy(x, x0, sizeof(float) * N); memcpy(y, y0, sizeof(float) * N); memcpy(z, z0, sizeof(float) * N);
  memcpy(vx, vx0, sizeof(float) * N); memcpy(vy, vy0, sizeof(float) * N); memcpy(vz, vz0, sizeof(float) * N);
  float* ax = (float*)malloc(sizeof(float) * 3 * (size_t)N);
  float *ay = ax + N, *az = ax + 2 * N;
  uint8_t* live = (uint8_t*)malloc((size_t)N);
  memset(live, 1, (size_t)N);
  double* x1 = (double*)malloc(sizeof(double) * n3 * (size_t)(T > 0 ? T : 1));
  double* m = (double*)malloc(sizeof(double) * N);
  double* vT = (double*)malloc(sizeof(double) * n3);
  for (int i = 0; i < N; ++i) m[i] = m32[i];
  const float h = 0.5f * dt;
  for (int s = 0; s < T; ++s) {
    for (int i = 0; i < N; ++i) {
      x[i] = x[i] + vx[i] * h; y[i] = y[i] + vy[i] * h; z[i] = z[i] + vz[i] * h;
      x1[n3 * s + 3 * i] = x[i]; x1[n3 * s + 3 * i + 1] = y[i]; x1[n3 * s + 3 * i + 2] = z[i];
    }
    orc_nbody_accel_f32(N, G, eps, x, y, z, m32, live, ax, ay, az);
    for (int i = 0; i < N; ++i) {
      vx[i] = vx[i] + ax[i] * dt; vy[i] = vy[i] + ay[i] * dt; vz[i] = vz[i] + az[i] * dt;
      x[i] = x[i] + vx[i] * h; y[i] = y[i] + vy[i] * h; z[i] = z[i] + vz[i] * h;
    }
  }
  double L = 0;
  for (int i = 0; i < N; ++i) {
    vT[3 * i] = vx[i]; vT[3 * i + 1] = vy[i]; vT[3 * i + 2] = vz[i];
    for (int c = 0; c < 3; ++c) L += 0.5 * m[i] * vT[3 * i + c] * vT[3 * i + c];
  }
  reverse_sweep(N, G, eps, dt, m, x1, T, vT, grad);
  if (loss) *loss = L;
  free(st); free(ax); free(live); free(x1); free(m); free(vT);
  return 0;
}

int orc_nbody_adjoint_f64(int N, double G, double eps, double dt,
                          const double* pos0, const double* vel0,
                          const double* m, int T, int ckpt, double* grad,
                          double* loss) {
  if (N < 1 || T < 0 || ckpt < 1) return -1;
  const size_t n3 = 3 * (size_t)N;
  const int nseg = (T + ckpt - 1) / ckpt;
  double* ck = (double*)malloc(sizeof(double) * 2 * n3 * (size_t)(nseg + 1));
  double* pos = (double*)malloc(sizeof(double) * n3);
  double* vel = (double*)malloc(sizeof(double) * n3);
  double* acc = (double*)malloc(sizeof(double) * n3);
  double* x1 = (double*)malloc(sizeof(double) * n3 * (size_t)ckpt);
  double* lx = (double*)calloc(n3, sizeof(double));
  double* lv = (double*)malloc(sizeof(double) * n3);
  double* w = (double*)malloc(sizeof(double) * n3);
  double* mu = (double*)malloc(sizeof(double) * n3);
  double* g = (double*)malloc(sizeof(double) * n3);
  memcpy(pos, pos0, sizeof(double) * n3);
  memcpy(vel, vel0, sizeof(double) * n3);
  /* forward pass, keeping (x, v) at the start of every segment */
  for (int s = 0; s < T; ++s) {
    if (s % ckpt == 0) {
      memcpy(ck + 2 * n3 * (size_t)(s / ckpt), pos, sizeof(double) * n3);
      memcpy(ck + 2 * n3 * (size_t)(s / ckpt) + n3, vel, sizeof(double) * n3);
    }
    step_f64(N, G, eps, dt, pos, vel, m, acc, NULL);
  }
  double L = 0;
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < 3; ++c) {
      L += 0.5 * m[i] * vel[3 * i + c] * vel[3 * i + c];
      lv[3 * i + c] = m[i] * vel[3 * i + c];
    }
  const double h = 0.5 * dt;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int s0 = seg * ckpt, s1 = (s0 + ckpt < T) ? s0 + ckpt : T;
    memcpy(pos, ck + 2 * n3 * (size_t)seg, sizeof(double) * n3);
    memcpy(vel, ck + 2 * n3 * (size_t)seg + n3, sizeof(double) * n3);
    for (int s = s0; s < s1; ++s)
      step_f64(N, G, eps, dt, pos, vel, m, acc, x1 + n3 * (size_t)(s - s0));
    for (int s = s1 - 1; s >= s0; --s) {
      for (size_t k = 0; k < n3; ++k) { w[k] = lv[k] + h * lx[k]; mu[k] = dt * w[k]; }
      orc_nbody_pair_adjoint_f64(N, G, eps, x1 + n3 * (size_t)(s - s0), m, mu, g);
      for (size_t k = 0; k < n3; ++k) { lx[k] += g[k]; lv[k] = w[k] + h * lx[k]; }
    }
  }
  memcpy(grad, lv, sizeof(double) * n3);
  if (loss) *loss = L;
  free(ck); free(pos); free(vel); free(acc); free(x1); free(lx); free(lv);
  free(w); free(mu); free(g);
  return 0;
}
