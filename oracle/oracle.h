/*
 * oracle.h -- CPU oracle for the SMMO hot path (TEST INFRASTRUCTURE ONLY).
 *
 * This is a plain, slow, array-of-structs restatement of the
 * SMMO workloads of the thesis (Springer, "Memory-Efficient
 * Object-Oriented Programming on GPUs", Ch. 7) plus its own Philox4x32-10.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load it.  It shares no code, header or constant generator with the CUDA
 * library in paper_1908_05845_gb300/csrc; the only thing both sides consume
 * in common are the seeded input arrays built by
 * paper_1908_05845_gb300/inputs.py, which contain none of the method's
 * arithmetic.
 *
 * Everything runs on one thread except the n-body receiver loops (FP32
 * forces and merge scan, FP64 forces and pair adjoint), which OpenMP may
 * spread over several: each receiver keeps its own partner order, so the
 * results do not depend on the thread count (orc_set_threads).
 *
 * Every entry point returns 0 on success and a negative value on bad
 * arguments.  All arrays are caller-owned host memory.
 */
#ifndef SMMO_ORACLE_H
#define SMMO_ORACLE_H
#include <stdint.h>

/* ---------------------------------------------------------------- Philox */
/* Philox4x32-10 block function (Salmon et al., SC'11, Sec. 3.2 / Table 2). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
/* draw(tag, step, cell, inst): word 0 of Philox4x32-10 with
 * key = (seed mod 2^32, seed >> 32), counter = (step, cell, tag, inst). */
uint32_t orc_draw(uint64_t seed, uint32_t tag, uint32_t step, uint32_t cell,
                  uint32_t inst);
void orc_draw_many(uint64_t seed, uint32_t tag, uint32_t step,
                   const uint32_t* cells, int64_t n, uint32_t inst,
                   uint32_t* out);

/* Random-stream tags used inside the method (step draws). */
enum {
  ORC_TAG_INIT = 0, ORC_TAG_FISH = 1, ORC_TAG_SHARK = 2, ORC_TAG_LEN = 3,
  ORC_TAG_PLACE = 4, ORC_TAG_ROUTE = 5, ORC_TAG_BRAKE = 6, ORC_TAG_KIND = 7,
  ORC_TAG_SIDE = 8, ORC_TAG_OUTDEG = 9, ORC_TAG_OUT = 10
};

/* ------------------------------------------------------------ Game of Life */
/* Cell kinds in the canonical per-cell output. */
enum { ORC_EMPTY = 0, ORC_ALIVE = 1, ORC_CANDIDATE = 2 };
/* Runs T generations of the object-based Life of Sec. 7.8 on a W x H torus.
 * kind/state: per-cell in/out arrays (kind: EMPTY/ALIVE/CANDIDATE; state:
 * is_new flag of an Alive object, 0 for candidates).  Per generation
 * counters (7 x int64 per generation, may be NULL):
 * [alive, candidates, births, deaths, candidates_created, candidates_deleted,
 *  allocs+frees]. */
int orc_gol_run(int W, int H, uint8_t* kind, uint8_t* state, int T,
                int64_t* counters);

/* ------------------------------------------- generational automaton */
/* Runs T generations of the "generation" extension of Life (Sec. 7.8):
 * survive/born are masks over the number of alive neighbours (bit n set =
 * survive / born with n), a dead Alive blocks its cell for `block`
 * generations before a Candidate replaces it (block 0 = Life semantics).
 * kind/state/blocked: per-cell in/out arrays (state: is_new of an Alive;
 * blocked: generations an Alive has blocked, 0 = alive).  counters (may be
 * NULL): 8 x int64 per generation: [alive, blocking, candidates, births,
 * deaths, expired, candidates_created, candidates_deleted]. */
int orc_gen_run(int W, int H, uint32_t survive, uint32_t born, int block,
                uint8_t* kind, uint8_t* state, uint16_t* blocked, int T,
                int64_t* counters);

/* ---------------------------------------------------------------- Wa-Tor */
enum { ORC_FISH = 1, ORC_SHARK = 2 };
typedef struct {
  int fish_breed, shark_breed, starve;
  int breed_strict; /* 0: breed when age >= breed (default); 1: age > breed */
} orc_wator_params;
/* Runs steps t0+1 .. t0+T of Wa-Tor (Sec. 7.6) on a W x H torus.
 * kind/age/energy are per-cell in/out arrays.  seed/inst select the draws.
 * counters (may be NULL): 8 x int64 per step:
 * [fish, sharks, fish_births, fish_eaten, shark_births, sharks_starved,
 *  fish_moves, shark_moves]. */
int orc_wator_run(int W, int H, uint64_t seed, uint32_t inst,
                  const orc_wator_params* p, int8_t* kind, int16_t* age,
                  int16_t* energy, int t0, int T, int64_t* counters);

/* ------------------------------------------------- Nagel-Schreckenberg */
typedef struct {
  int num_streets;
  const int32_t* street_start; /* first cell of each street */
  const int32_t* street_len;   /* length (cells) of each street */
  const int32_t* out_deg;      /* number of outgoing streets (0 = sink) */
  const int32_t* out_street;   /* num_streets x 3 outgoing street ids */
  const uint8_t* is_source;    /* 1 = spawns cars at its first cell */
  int num_cells;
  int v_max;
  uint32_t brake_threshold;    /* floor(p * 2^32) */
  int sources_enabled;         /* 0 disables car creation */
  int sinks_enabled;           /* 0 keeps cars on sink streets (blocked) */
} orc_nasch_graph;
/* car_v: per-cell in/out array, -1 = no car, else velocity.
 * counters (may be NULL): 4 x int64 per step: [cars, spawned, sunk, moved]. */
int orc_nasch_run(const orc_nasch_graph* g, uint64_t seed, int8_t* car_v,
                  int t0, int T, int64_t* counters);

/* Traffic controllers (Sec. 7.5): per street o, ctrl_kind[o] = -1 (none),
 * 0 traffic light, 1 smart traffic light, 2 yield controller; a controller
 * acts only when o has two or more incoming streets. */
enum { ORC_CTRL_LIGHT = 0, ORC_CTRL_SMART = 1, ORC_CTRL_YIELD = 2 };
typedef struct {
  const int8_t* ctrl_kind;
  int phase_len;  /* green phase of a traffic light, steps (>= 1) */
  int lookahead;  /* cells before a crossing checked for a waiting car */
} orc_nasch_ctrl;
/* Runs steps t0+1 .. t0+T of traffic with controllers.  car_v as in
 * orc_nasch_run; green/timer: per-street in/out controller state (index of
 * the green incoming street, phase timer).  counters (may be NULL): 6 x
 * int64 per step: [cars, spawned, sunk, moved, claims_lost, switches]. */
int orc_nasch_ctrl_run(const orc_nasch_graph* g, const orc_nasch_ctrl* ctl,
                       uint64_t seed, int8_t* car_v, int16_t* green,
                       int16_t* timer, int t0, int T, int64_t* counters);

/* ----------------------------------------------------------------- BFS */
/* Distances from `source` on a CSR graph (row_ptr: n + 1 offsets, col:
 * neighbours); INT32_MAX = unreachable; *levels = largest distance + 1. */
int orc_bfs(int n, const int32_t* row_ptr, const int32_t* col, int source,
            int32_t* dist, int* levels);

/* ---------------------------------------------------------- Barnes-Hut */
typedef struct {
  float G, eps, dt, theta;
} orc_bh_params;
/* 2-D Barnes-Hut (Sec. 7.3) on the unit square, FP32 with the fixed order
 * given in barnes_hut.c.  x, y, vx, vy: N-long in/out; m: masses.
 * counters (may be NULL): 2 x int64 per step: [tree nodes, node visits].
 * Returns -1 on bad arguments or two bodies at the same position. */
int orc_bh_run(int N, const orc_bh_params* p, float* x, float* y, float* vx,
               float* vy, const float* m, int T, int64_t* counters);
/* Accelerations (without G) of one tree build, same arithmetic. */
int orc_bh_accel(int N, float eps, float theta, const float* x, const float* y,
                 const float* m, float* ax, float* ay);
/* Tree-node count and depth of the region quad tree of the positions. */
int orc_bh_build(int N, const float* x, const float* y, int* nodes, int* depth);

/* ---------------------------------------------------------------- N-body */
typedef struct {
  float G, eps, dt, merge_r;
  int merge; /* 1: collision merge after each step */
} orc_nbody_params_f32;
/* FP32 DKD leapfrog with fixed evaluation order.  Arrays are N-long, indexed
 * by body id; live[i] = 0 marks a body freed by a merge.  counters: 1 x
 * int64 per step (merges in that step).  */
int orc_nbody_run_f32(int N, const orc_nbody_params_f32* p, float* x, float* y,
                      float* z, float* vx, float* vy, float* vz, float* m,
                      uint8_t* live, int T, int64_t* counters);
/* Threads for the n-body receiver loops (n <= 0: OpenMP's default);
 * returns the count now in use (1 when built without OpenMP). */
int orc_set_threads(int n);
/* Accelerations only (one force evaluation), FP32, same order as the run. */
int orc_nbody_accel_f32(int N, float G, float eps, const float* x,
                        const float* y, const float* z, const float* m,
                        const uint8_t* live, float* ax, float* ay, float* az);

/* One no-merge FP32 step for the listed receivers only (out: 6 floats per
 * listed body: x, y, z, vx, vy, vz after the step), same arithmetic. */
int orc_nbody_step_sample_f32(int N, float G, float eps, float dt, const float* x,
                              const float* y, const float* z, const float* vx,
                              const float* vy, const float* vz, const float* m,
                              const uint8_t* live, const int32_t* idx, int nidx,
                              float* out);

/* FP64 variants (no merge).  pos/vel: N x 3 row-major. */
int orc_nbody_run_f64(int N, double G, double eps, double dt, double* pos,
                      double* vel, const double* m, int T);
int orc_nbody_accel_f64(int N, double G, double eps, const double* pos,
                        const double* m, double* acc);
/* Energy E = KE - G sum_{i<j} m_i m_j / sqrt(r^2 + eps^2), momentum P. */
int orc_nbody_energy_f64(int N, double G, double eps, const double* pos,
                         const double* vel, const double* m, double* E,
                         double* P3);
/* Adjoint of the no-merge DKD run: gradient of L = 1/2 sum m |v_T|^2 with
 * respect to the initial velocities, checkpointing (x, v) every `ckpt`
 * steps and recomputing within each segment.  grad: N x 3.  loss: L. */
int orc_nbody_adjoint_f64(int N, double G, double eps, double dt,
                          const double* pos0, const double* vel0,
                          const double* m, int T, int ckpt, double* grad,
                          double* loss);
/* FP64 reverse sweep along the FP32 no-merge trajectory (forward pass as in
 * orc_nbody_run_f32, mid-step positions and final velocities widened to
 * double).  grad: N x 3. */
int orc_nbody_adjoint_f32traj(int N, float G, float eps, float dt, const float* x0,
                              const float* y0, const float* z0, const float* vx0,
                              const float* vy0, const float* vz0, const float* m32,
                              int T, double* grad, double* loss);
/* One application of the pair kernel g_k = G sum_{j!=k} H(x_j - x_k)
 * (m_k mu_j - m_j mu_k), H(r) = I/s^3 - 3 r r^T / s^5. */
int orc_nbody_pair_adjoint_f64(int N, double G, double eps, const double* pos,
                               const double* m, const double* mu, double* g);

/* ------------------------------------------------------------ structure */
/* Spring mesh with cracks (Sec. 7.4); the arithmetic and order are given
 * in structure.c.  Node kinds: */
#define ORC_STRUCT_ANCHOR 0
#define ORC_STRUCT_PULL 1
#define ORC_STRUCT_NODE 2
/* phases of one iteration (bit mask; 7 = all) */
#define ORC_STRUCT_PHASE_PULL 1
#define ORC_STRUCT_PHASE_COMPUTE 2
#define ORC_STRUCT_PHASE_REMOVE 4
typedef struct {
  float dt, damping;
  int32_t substeps;
} orc_structure_params;
/* Nodes 0..N-1: kind, position x/y, velocity vx/vy (constant for pull
 * nodes), mass m, slot (3 N spring ids, -1 empty), nspr (springs held),
 * nalive.  Springs 0..S-1: endpoints p1/p2, stiffness k, rest length L0,
 * break limit fmax, force on p1 fx/fy, salive.  dist: distances of the
 * last removal phase (INT32_MAX unreached).  Arrays are updated in place.
 * counters (may be NULL): 5 x int64 per iteration: springs broken, nodes
 * deleted by breaks, springs deleted by the removal, nodes deleted by the
 * removal, BFS levels run. */
int orc_structure_run(int N, int S, const orc_structure_params* p, const int8_t* kind,
                      float* x, float* y, float* vx, float* vy, const float* m,
                      int32_t* slot, int32_t* nspr, uint8_t* nalive, const int32_t* p1,
                      const int32_t* p2, const float* k, const float* L0,
                      const float* fmax, float* fx, float* fy, uint8_t* salive,
                      int32_t* dist, int T, int phases, int64_t* counters);

#endif
