/*
 * smmo.h -- C ABI of the GB300 SMMO heap ("Single-Method Multiple-Objects":
 * run one method on every live object of a class, objects stored in a
 * Structure-of-Arrays heap with a device-side allocator).
 *
 * Thesis: M. Springer, "Memory-Efficient Object-Oriented Programming on
 * GPUs" (arXiv 1908.05845).  Citations below name its sections, equations
 * and algorithms.
 *
 * General rules
 *  - Every call returns an int status (SMMO_OK = 0 or a negative SMMO_E_*).
 *  - Pointers documented as "device" must point to device memory of the
 *    current CUDA device; "host" pointers to host memory.  The library never
 *    frees memory it did not allocate; caller-owned buffers stay
 *    caller-owned.
 *  - `stream` arguments are cudaStream_t values passed as void* (0 = the
 *    legacy default stream).  Calls documented as asynchronous only enqueue
 *    work; device-side failures (heap exhausted during a device `new`, a
 *    retry budget running out, a double free) are recorded in the heap's
 *    device error word and reported by smmo_heap_sync().
 *  - A heap must be used from one stream at a time (its enumeration scratch
 *    is shared by consecutive parallel_do calls).
 *  - Device loops never spin without bound: every retry loop has a budget
 *    and sets SMMO_E_CONTENTION or SMMO_E_DEVICE_OOM when it runs out.
 */
#ifndef SMMO_H
#define SMMO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status */
enum {
  SMMO_OK = 0,
  SMMO_E_INVALID_ARG = -1,  /* bad argument (null pointer, id out of range) */
  SMMO_E_OOM = -2,          /* heap has too few free blocks (host check)    */
  SMMO_E_DEVICE_OOM = -3,   /* a device `new` found no free block            */
  SMMO_E_CONTENTION = -4,   /* a device retry budget ran out                 */
  SMMO_E_CUDA = -5,         /* a CUDA runtime call failed; see last_cuda_error */
  SMMO_E_TIMEOUT = -6,      /* host wait exceeded its limit                  */
  SMMO_E_BAD_HANDLE = -7,   /* double free / foreign handle                  */
  SMMO_E_BOUNDS = -8,       /* debug bounds check failed                     */
  SMMO_E_UNSUPPORTED = -9,  /* operation not supported in this state         */
  SMMO_E_FROZEN = -10       /* class registration after the first bulk_new   */
};

const char* smmo_status_string(int status);
/* Last CUDA error code observed by the library (cudaError_t as int). */
int smmo_last_cuda_error(void);

/* -------------------------------------------------------------- types */
typedef struct smmo_heap smmo_heap;

/* Handle of an object: (block index << 6) | slot.  0xFFFFFFFF = null.
 * Replaces the thesis' 64-bit "fake pointer" (Sec. 5.2.3: block address,
 * slot in bits 0-5, capacity and type id in the high bits); the type id
 * and capacity are looked up in per-block and per-class tables instead. */
typedef uint32_t smmo_handle;
#define SMMO_NULL_HANDLE 0xFFFFFFFFu

enum {
  SMMO_I8 = 1, SMMO_U8 = 2, SMMO_I16 = 3, SMMO_U16 = 4, SMMO_I32 = 5,
  SMMO_U32 = 6, SMMO_F32 = 7, SMMO_I64 = 8, SMMO_U64 = 9, SMMO_F64 = 10,
  SMMO_HANDLE = 11, /* a smmo_handle (4 bytes) */
  /* uint32 index of the object's instance in the heap's instance table
   * (smmo_batch_define); bulk_new records SMMO_E_BOUNDS for an index
   * outside the table */
  SMMO_INSTANCE = 12
};

#define SMMO_MAX_CLASSES 16
#define SMMO_MAX_FIELDS 16

/* One field of a class.  `count` > 1 declares a fixed-length inner array
 * stored as `count` separate SOA columns ("SOA, full inlining", Sec. 4.3).
 * `ref_class` names the class a SMMO_HANDLE field refers to (-1 = unknown);
 * compaction of class T rewrites every HANDLE column whose ref_class is T
 * or a superclass of T (Sec. 6.3.5, "limiting heap scans"). */
typedef struct {
  const char* name;
  int elem_type;
  int count;
  int ref_class;
} smmo_field_desc;

typedef struct {
  /* Bytes of a block's data segment.  0 = 64 * size of the smallest
   * registered class (Sec. 5.2.2, block capacity
   * N_T = floor(64 size(T_s) / size(T))). Rounded up to 64. */
  uint32_t block_data_bytes;
  /* Active-block lookups tried before a new block is initialised
   * (Sec. 5.3.2, "lookup retry").  Default 5. */
  int32_t lookup_retries;
  /* Budget of a device `new` (rounds of warp-aggregated reservation) and
   * of bitmap spin loops.  Defaults 4096 and 1 << 20. */
  int32_t alloc_retries;
  int32_t bitmap_spins;
  /* parallel_do launch shape: threads per CTA (multiple of 64, at most
   * 512) and CTAs per SM of the persistent grid.  Defaults 256 and 8. */
  int32_t threads_per_cta;
  int32_t ctas_per_sm;
  /* 1 = device code checks handles and indices and records the first
   * violation as SMMO_E_BOUNDS instead of touching memory. */
  int32_t debug_checks;
  /* n of the defragmentation-candidate state kept by new and delete
   * (Sec. 6.3.1): a block is a candidate iff it holds at most
   * floor(N_T n / (n + 1)) objects.  Warp caches refill from candidates
   * first.  Default 1 (at most half full). */
  int32_t defrag_factor;
  /* Fan-out of the hierarchical bitmaps (Sec. 5.3.1): bits per container,
   * 32 or 64 (default 64).  A container of 32 is half of a 64-bit word, so
   * level 0 is stored the same way for both; with 32 every level above
   * has one bit per 32 bits below it (one more level for large heaps, a
   * lookup descends a narrower word). */
  int32_t bitmap_fanout;
} smmo_heap_config;

/* Fills `cfg` with the defaults above. */
void smmo_heap_config_default(smmo_heap_config* cfg);

typedef struct {
  int64_t live_objects[SMMO_MAX_CLASSES];  /* per class (not subclasses) */
  int64_t blocks[SMMO_MAX_CLASSES];        /* allocated blocks per class  */
  int64_t free_blocks;
  int64_t num_blocks;                       /* M                          */
  double fragmentation[SMMO_MAX_CLASSES];   /* F of Sec. 6.2.2, per class */
  double fragmentation_all;                 /* F over all allocated blocks */
  int64_t allocs[SMMO_MAX_CLASSES];         /* device news since create   */
  int64_t frees[SMMO_MAX_CLASSES];          /* device deletes since create */
  int64_t slow_paths;                       /* blocks initialised by news */
  int64_t enumerated_objects;               /* objects visited by do-alls */
  int64_t enumerated_blocks;
  int32_t capacity[SMMO_MAX_CLASSES];       /* N_T per class              */
  int32_t object_bytes[SMMO_MAX_CLASSES];
  int32_t block_bytes;
  int32_t num_classes;
} smmo_heap_stats;

typedef struct {
  int32_t passes;             /* defragmentation passes run              */
  int64_t blocks_freed;       /* source blocks eliminated                */
  int64_t objects_moved;
  int64_t pointers_rewritten;
  int64_t candidates_left;    /* candidates after the last pass          */
  /* device time of the phases (CUDA events on the stream), summed over
   * passes: candidate scan and sorted list; object copy and forwarding
   * pointers; block-state update; and the final pointer rewrite (with its
   * enumeration of each referring class) */
  double scan_ms;
  double copy_ms;
  double state_ms;
  double rewrite_ms;
} smmo_compact_stats;

/* ------------------------------------------------------------- heap */
/* Creates a heap inside the caller's device buffer (Sec. 5.2: one heap of
 * M equal-size blocks; Sec. 5.3.1 hierarchical bitmaps).  The heap borrows
 * `dev_buf` (>= 1 MiB, 256-byte aligned) and never frees it; the buffer
 * must outlive the heap.  `cfg` may be NULL (defaults).  The block geometry
 * is fixed when the first object is created. */
int smmo_heap_create(const smmo_heap_config* cfg, void* dev_buf,
                     size_t buf_bytes, void* stream, smmo_heap** out);
/* Releases the host-side heap object and the small device state the
 * library allocated; does not touch `dev_buf`. */
int smmo_heap_destroy(smmo_heap* heap);

/* Registers a class (Sec. 5.1.1 "Data Layout DSL", "Class Inheritance").
 * Inherited fields come first (field i of the parent is field i of the
 * child).  Abstract classes own no objects; parallel_do on them runs every
 * concrete subclass.  Must precede the first bulk_new (SMMO_E_FROZEN). */
int smmo_class_register(smmo_heap* heap, const char* name,
                        const smmo_field_desc* fields, int nfields,
                        int parent_class, int is_abstract, int* class_id);
int smmo_class_lookup(smmo_heap* heap, const char* name, int* class_id);
/* Number of fields (including inherited) and capacity N_T of a class;
 * valid after the geometry is fixed (first bulk_new or smmo_heap_freeze). */
int smmo_class_info(smmo_heap* heap, int class_id, int* nfields,
                    int* capacity, int* object_bytes);
/* Fixes the block geometry now (otherwise done by the first bulk_new). */
int smmo_heap_freeze(smmo_heap* heap);

/* Methods are compiled into the library and looked up by name, e.g.
 * "test.add_i32", "wator.fish_prepare" (see the workload sections); the
 * thesis' methods are members of the classes (Sec. 5.1.1), here they are
 * kernels that take the class as an argument.  heap may be NULL (the id
 * is the same for every heap); with a heap whose geometry is fixed, a
 * method that needs a batch (the test.batch_* methods) is rejected
 * (SMMO_E_UNSUPPORTED) when the heap has no instance table. */
int smmo_method_lookup(smmo_heap* heap, const char* name, int* method_id);

/* ----------------------------------------------------------- batches
 * A batch is a set of independent problem instances whose objects share
 * one heap: one parallel_do of a class runs the method on the objects of
 * every instance in a single launch (the thesis' parallel_do, Sec. 5.2.7,
 * over all objects of a class, whatever instance they belong to).  The
 * instance table is owned by the heap and lives in its buffer; an object
 * names its instance in a SMMO_INSTANCE field, and a method reads the
 * instance's row through the heap (device code: smmo::instance_of).
 * Instances that own a range of a global numbering (the cells of the
 * cellular worlds) can also be found from an index in their range. */
typedef struct {
  int32_t kind;      /* caller-defined kind (the worlds: SMMO_WORLD_*)     */
  uint32_t id;       /* the instance's number in its random counters       */
  uint32_t W, H;     /* grid extent (0 when the instance has no grid)      */
  uint64_t base;     /* first index of its range of a global numbering     */
  uint64_t count;    /* length of that range (0: none)                     */
  int64_t param[2];  /* caller-defined parameters                          */
} smmo_instance_desc;
/* Gives the heap its instance table: n_inst (1 .. 2^20) rows, copied (host
 * array `inst`).  Ranges [base, base + count) must ascend and not overlap,
 * and end below 2^32.  Must precede the first bulk_new / freeze (else
 * SMMO_E_FROZEN); once per heap.  The table is carved from the heap
 * buffer when the geometry is fixed. */
int smmo_batch_define(smmo_heap* heap, const smmo_instance_desc* inst, int n_inst);
/* Instances in the heap's table (0: none) into *n_inst (host). */
int smmo_batch_count(smmo_heap* heap, int* n_inst);

/* Host-launched creation of n objects of a concrete class (the thesis'
 * parallel_new, Sec. 5.1.1).  field_src[k] is a device array of n elements
 * for SOA column k (columns are the fields in order, an inner array of
 * `count` elements contributing `count` columns).  Objects fill whole free
 * blocks in ascending block order; out_handles (device, nullable) receives
 * their handles.  Asynchronous on `stream` (capturable) unless
 * out_first_block is given: then it synchronises `stream` and writes the
 * first block index when the blocks used are consecutive, else -1 (objects
 * i then sit at block first + i / N_T, slot i % N_T).  Fixing the geometry
 * (the first bulk_new of a heap) also synchronises.  SMMO_E_OOM at once if
 * ceil(n / N_T) exceeds the heap's block count; if fewer blocks are free
 * when the kernels run, nothing is created and SMMO_E_OOM is recorded in
 * the device error word (smmo_heap_sync; synchronous calls return it). */
int smmo_bulk_new(smmo_heap* heap, int class_id, int64_t n,
                  const void* const* field_src, smmo_handle* out_handles,
                  int64_t* out_first_block, void* stream);

/* parallel_do(class, method) (Sec. 5.2.7): for every concrete class C in
 * the subtree of `class_id`, snapshot the allocated blocks of C with their
 * allocation bitmaps, then run `method` once for every object of C that
 * existed at that point, one thread per slot.  Objects created by the
 * method are not visited; the method may delete only its own object of
 * the visited class (and any object of another class).  `args` (host,
 * args_bytes <= 1024) is copied by value into the kernel parameters.
 * Asynchronous; capturable in a CUDA graph. */
int smmo_parallel_do(smmo_heap* heap, int class_id, int method_id,
                     const void* args, size_t args_bytes, void* stream);

/* Reducers of smmo_parallel_do_and_reduce (64-bit signed integers; sum
 * wraps). */
enum {
  SMMO_REDUCE_SUM = 0,
  SMMO_REDUCE_MIN = 1,
  SMMO_REDUCE_MAX = 2,
  SMMO_REDUCE_OR = 3,
  SMMO_REDUCE_AND = 4
};
/* parallel_do_and_reduce (Sec. 3.2.2): runs reducing method method_id (one
 * whose per-object result is an int64) on every object of class_id and its
 * concrete subclasses that exists at invocation, and combines the results
 * with reducer `op` into *dev_result (a device int64 owned by the caller;
 * it is set to the reducer's identity first, so no object gives the
 * identity).  Same object semantics and argument rules as
 * smmo_parallel_do; SMMO_E_INVALID_ARG if the method does not reduce.
 * Asynchronous (capturable in a CUDA graph). */
int smmo_parallel_do_and_reduce(smmo_heap* heap, int class_id, int method_id,
                                const void* args, size_t args_bytes, int op,
                                int64_t* dev_result, void* stream);

/* Handles of all live objects of class_id (and of its subclasses when
 * include_subclasses != 0), in unspecified order, into out_handles
 * (device, capacity `cap`).  *out_count (host) receives the full count,
 * which may exceed cap (output truncated).  Synchronises `stream`.  The
 * enumeration follows the thesis' indices() of the allocated-block bitmaps
 * (Sec. 5.3.1, "enumerating set bit indices"). */
int smmo_enumerate_live(smmo_heap* heap, int class_id, int include_subclasses,
                        smmo_handle* out_handles, int64_t cap,
                        int64_t* out_count, void* stream);

/* Copies field columns of n objects into dense arrays: dst[k][i] = column
 * `columns[k]` of object handles[i], read from the SOA columns of the
 * objects' blocks (block structure, Sec. 5.2.1).  Column indices count
 * inner-array columns (see bulk_new).  handles/dst are device pointers;
 * `columns` and `dst` arrays are host arrays of length ncol.
 * Asynchronous. */
int smmo_gather_fields(smmo_heap* heap, int class_id, const smmo_handle* handles,
                       int64_t n, const int* columns, int ncol,
                       void* const* dst, void* stream);

/* Defragments class_id (CompactGpu, Ch. 6): passes of (1) candidate scan
 * (blocks at most n/(n+1) full, Sec. 6.3.1), (2) source/target assignment
 * (first B = floor(r/(n+1)) candidates are sources, Sec. 6.3.3), (3) object
 * copy, (4) forwarding pointers in the source blocks, (5) block-state
 * update, until at most k1 candidates remain (Sec. 6.3.7); then (6) one
 * rewrite of every HANDLE column that may refer to class_id (ref_class
 * class_id, a superclass of it, or -1), following forwarding pointers
 * through all passes (Alg. 6.6; the thesis rewrites after each pass, with
 * the same result).  n in 1..63, k1 >= 0.  Handles held outside the heap
 * are invalidated.  Allocates nothing (its scratch is part of the heap
 * buffer).  Synchronises `stream`. */
int smmo_compact(smmo_heap* heap, int class_id, int defrag_factor,
                 int64_t k1, smmo_compact_stats* out, void* stream);

/* Rewrites n caller-held handles (device array) to where the last
 * smmo_compact moved their objects (following its forwarding slots,
 * Sec. 6.3.4, as the rewrite of the heap's own HANDLE columns does,
 * Sec. 6.3.5; handles of objects that did not move are unchanged).  Valid until the next allocation: returns
 * SMMO_E_UNSUPPORTED once a device new or bulk_new has run since that
 * compaction (the freed source blocks may hold new objects).  Synchronises
 * `stream`. */
int smmo_remap_handles(smmo_heap* heap, smmo_handle* handles, int64_t n, void* stream);

/* Number of defragmentation candidates of class_id for factor n (allocated
 * blocks holding at most floor(N_T n / (n + 1)) objects, Sec. 6.3.1) into
 * *count (host).  Synchronises `stream`. */
int smmo_defrag_candidates(smmo_heap* heap, int class_id, int defrag_factor,
                           int64_t* count, void* stream);

/* The "after massive deallocations" policy of Sec. 6.3.8: compacts class_id
 * (as smmo_compact with n = defrag_factor and k1) iff its candidate count
 * is at least k2 n / (n + 1), where k2 = max(k2_blocks, k2_fraction x the
 * heap's block count M) (k2_fraction in [0, 1]).  *ran (host, nullable) =
 * 1 if it compacted; when it did not, *out holds zeros except
 * candidates_left = the count.  Synchronises `stream`.  (The other policy,
 * every m iterations, is a loop in the caller.) */
int smmo_compact_if(smmo_heap* heap, int class_id, int defrag_factor, int64_t k1,
                    int64_t k2_blocks, double k2_fraction, smmo_compact_stats* out,
                    int* ran, void* stream);

/* Statistics (Sec. 6.2.2 fragmentation F; device counters).  Synchronises
 * `stream`. */
int smmo_heap_get_stats(smmo_heap* heap, smmo_heap_stats* out, void* stream);

/* Checks the heap invariants after all kernels have finished (Sec. 5.4.5,
 * consistency of hierarchical bitmaps; Sec. 6.2.2, block states):
 * every higher-level bit equals the OR of its container; a block is either
 * free or allocated to exactly one class, the one in its type id; a block
 * is active iff it is allocated and not full; an allocated block holds at
 * least one object; free blocks have no object.  *violations (host)
 * receives the number of violated checks (0 = consistent).  Synchronises
 * `stream`. */
int smmo_heap_check(smmo_heap* heap, int64_t* violations, void* stream);

/* Cumulative device counters since create: objects visited by do-all
 * kernels (every object a method ran on, counted per launch), device news
 * and device deletes (all classes).  Host outputs (nullable).  Synchronises
 * `stream`; reads the 10 KB counter array. */
int smmo_heap_counters(smmo_heap* heap, int64_t* enumerated_objects,
                       int64_t* allocs, int64_t* frees, void* stream);

/* Cumulative allocator event counters (host array of 6): blocks
 * initialised by the slow path, allocation rounds retried, warp-cache
 * refills, active-block lookups that found nothing, reservations that found
 * the chosen block full, blocks enumerated.  Synchronises `stream`. */
int smmo_heap_alloc_counters(smmo_heap* heap, int64_t* out6, void* stream);

/* Synchronises `stream` and reads the first device error recorded since the
 * last smmo_heap_sync without clearing it: *code (host) = the status (0 =
 * none), *detail (host, nullable) = its detail word. */
int smmo_heap_last_device_error(smmo_heap* heap, int* code, uint64_t* detail, void* stream);

/* Synchronises `stream` and returns the first device error recorded since
 * the last sync (then clears it).  *detail (host, nullable) receives the
 * error's detail word (e.g. the offending handle).  For SMMO_E_CONTENTION,
 * bits 48..55 name the loop that gave up: 1 propagation of a hierarchical
 * bitmap bit (bits 32..47 the bitmap, 0..31 the position), 2 / 3 a blocking
 * bitmap set / clear (same fields), 4 the block-state updates of a
 * deallocation (bits 32..47 the pending active, allocated, free and
 * candidate changes, 4 bits each, two's complement; bits 0..31 the block),
 * 5 the warp allocation cache's lock, 6 the rounds of a device new (bits
 * 0..31 the class); 0 a workload's own site (see its section).  Device retry loops are
 * bounded and record SMMO_E_CONTENTION / SMMO_E_DEVICE_OOM here where the
 * thesis' allocation retries without bound (Alg. 5.1). */
int smmo_heap_sync(smmo_heap* heap, void* stream, uint64_t* detail);

/* Device pointer to the start of a block's data segment and the column
 * offset table of a class, for callers writing their own kernels.
 * col_off (host, SMMO_MAX_FIELDS*?) receives per-column byte offsets inside
 * a block; *block_bytes the block stride. */
int smmo_class_layout(smmo_heap* heap, int class_id, uint32_t* col_off,
                      int* ncols, uint32_t* block_bytes, void** data_base);

/* ===================================================== cellular workloads
 * A "world" is a set of independent simulation instances of the thesis'
 * cellular SMMO applications on one heap (Ch. 7): object-based Game of Life
 * (Sec. 7.8; classes Cell, LAgent, Alive, Candidate) and Wa-Tor (Sec. 7.6;
 * classes Cell, WAgent, Fish, Shark), each on its own W x H torus.  All
 * instances' objects share the heap; one step runs every do-all of the
 * step once per class over all instances (one Life generation and one
 * Wa-Tor iteration).  With one instance this is the plain single
 * simulation.  Randomness is Philox4x32-10 keyed by
 * (seed; step, local cell, tag, instance); contested cells go to the agent
 * on the lowest cell index. */
typedef struct smmo_world smmo_world;
enum { SMMO_WORLD_LIFE = 0, SMMO_WORLD_WATOR = 1 };

typedef struct {
  int fish_breed;   /* fish breed when age >= fish_breed (default 4)   */
  int shark_breed;  /* sharks likewise (default 12)                    */
  int starve;       /* shark energy after eating / at birth (3)        */
  int breed_strict; /* 1: breed when age > breed instead of >=         */
} smmo_wator_params;

/* Registers the classes in a fresh heap (no class registered yet, else
 * SMMO_E_FROZEN), gives the heap its instance table (smmo_batch_define:
 * instance i has kind[i], W[i] x H[i] cells starting at the sum of the
 * sizes before it, and draws with instance number i) and creates the
 * instances.  kind/W/H: host arrays of n_inst entries (W, H >= 3; at most
 * 2^30 - 2 cells in all).
 * Per-cell initial state: device arrays over
 * the concatenation of all instances' cells in instance order, row-major
 * (cell = y * W + x): init_kind (Life: 0 empty, 1 Alive, 2 Candidate;
 * Wa-Tor: 0 empty, 1 Fish, 2 Shark), init_age (Wa-Tor: age; Life: the
 * generations an Alive has blocked its cell, 0 = alive; nullable = 0),
 * init_energy (Wa-Tor, nullable = 0), init_state (Life is_new flag,
 * nullable = 0).  params may be NULL.  Life-kind instances start with the
 * Life rule (see smmo_world_set_life_rule).  Synchronises `stream`.  The
 * world allocates its 4-byte step counter with cudaMalloc, freed by
 * smmo_world_destroy (with 1 KiB of grid-barrier words behind it), and,
 * when there are Wa-Tor instances, a creation queue of 4.125 bytes per cell
 * plus 132 bytes per warp slot of the GPU (also cudaMalloc). */
int smmo_world_create(smmo_heap* heap, int n_inst, const int* kind,
                      const uint32_t* W, const uint32_t* H, uint64_t seed,
                      const smmo_wator_params* params, const int8_t* init_kind,
                      const int16_t* init_age, const int16_t* init_energy,
                      const uint8_t* init_state, void* stream,
                      smmo_world** out);
/* As smmo_world_create with the instance table given as rows (host array
 * of n_inst): kind, id (the instance number of its draws, any value, so
 * one instance of a larger batch can be run alone with its own draws), W
 * and H are used; base and count must be the running sum of the sizes
 * and W x H (else SMMO_E_INVALID_ARG); param is ignored. */
int smmo_world_create_batch(smmo_heap* heap, const smmo_instance_desc* inst, int n_inst,
                            uint64_t seed, const smmo_wator_params* params,
                            const int8_t* init_kind, const int16_t* init_age,
                            const int16_t* init_energy, const uint8_t* init_state,
                            void* stream, smmo_world** out);
/* Advances every instance by nsteps steps.  Asynchronous (host loop of
 * parallel_do launches; capturable in a CUDA graph). */
int smmo_world_step(smmo_world* w, int nsteps, void* stream);
/* Rule of the Life-kind instances (Sec. 7.8, "gol" and its "generation"
 * extension): with n = alive Alive objects among the 8 neighbours (a dead
 * Alive that blocks its cell does not count), an Alive survives iff bit n
 * of `survive` is set, a Candidate becomes a new Alive iff bit n of `born`
 * is set; a dead Alive keeps its cell blocked for `block` generations and
 * is then replaced by a Candidate (block 0: replaced at once).  Life:
 * survive 0x00C, born 0x008, block 0 (the default); Burst: survive 0x1ED,
 * born 0x158, block 255.  survive, born < 2^9 (born bit 0 is invalid: a
 * Candidate without alive neighbour is deleted), block <= 65535.  Takes
 * effect at the next step; drops a captured graph. */
int smmo_world_set_life_rule(smmo_world* w, uint32_t survive, uint32_t born, uint32_t block);
/* How a Wa-Tor iteration (Sec. 7.6: every agent of a species posts its
 * move request, then every agent reads the requests and moves) is
 * launched; the results are the same in every mode.
 *   SMMO_WATOR_FOUR_DO_ALLS (the default): parallel_do(Fish, prepare), parallel_do(Fish,
 *     update), then the same for Shark: four do-all launches, the request
 *     word passed through the agent's target field.
 *   SMMO_WATOR_PHASED1 / SMMO_WATOR_PHASED2: each species'
 *     prepare and update in one cooperative launch over one snapshot, the
 *     phases separated by a grid barrier, the request word kept in shared
 *     memory between them; 1 or 2 units of 32 slots per warp round.
 *   | SMMO_WATOR_QUEUED_CREATION (with any of the above): the newborns of
 *     an update are written to a queue (payload and placement hint) instead
 *     of being allocated inside the update, and one more launch after it
 *     creates them, a full warp per 32.
 *   | SMMO_WATOR_MARKED_UPDATE (with SMMO_WATOR_FOUR_DO_ALLS only): the
 *     prepare do-all marks, per 32 slots, the agents that posted a request
 *     (or starve), and the update do-all runs its method only on those; it
 *     still walks and counts every agent.
 * Any other value: SMMO_E_INVALID_ARG.  Takes effect at the next step;
 * drops a captured graph. */
enum { SMMO_WATOR_FOUR_DO_ALLS = 0, SMMO_WATOR_PHASED1 = 1, SMMO_WATOR_PHASED2 = 2,
       SMMO_WATOR_QUEUED_CREATION = 4, SMMO_WATOR_MARKED_UPDATE = 8 };
int smmo_world_set_step_kernels(smmo_world* w, int mode);
/* Writes the live objects into per-cell device arrays (same indexing as
 * the initial state; kind, age, energy, state as above, age of an Alive =
 * its blocked count; empty cells 0) and
 * counts consistency errors (two agents on a cell, a cell not pointing back
 * at its agent) into *errors (host, nullable).  Synchronises `stream`. */
int smmo_world_export(smmo_world* w, int8_t* kind, int16_t* age, int16_t* energy,
                      uint8_t* state, int64_t* errors, void* stream);
/* Captures nsteps steps of the world into a CUDA graph (the step counter
 * lives in device memory, so every replay advances the simulation by
 * nsteps steps).  `stream` must be a non-default stream; nothing runs
 * during the capture.  smmo_world_replay launches the graph on `stream`
 * (asynchronous). */
int smmo_world_capture(smmo_world* w, int nsteps, void* stream);
int smmo_world_replay(smmo_world* w, void* stream);
/* As smmo_world_step, and additionally records CUDA events on `stream`
 * around every enumeration and do-all kernel and adds their durations (ms)
 * to phase_ms (host, 16 doubles, accumulated): index 2*p is the
 * enumeration and 2*p+1 the method kernel of phase p = Life candidate
 * prepare, alive prepare, candidate update, alive update, fish prepare,
 * fish update, shark prepare, shark update (in the fused modes of
 * smmo_world_set_step_kernels the fish and shark prepare phases p = 4 and 6
 * hold the fused launch, and p = 5 and 7 stay 0).  step_ms (host, nullable)
 * accumulates the device time from the first to the last launch of each
 * step; launches (host, nullable) is increased by the number of kernels
 * launched.  Synchronises `stream` once, after the last step. */
int smmo_world_step_profiled(smmo_world* w, int nsteps, double* phase_ms,
                             double* step_ms, int64_t* launches, void* stream);
/* Allocation-free variant of smmo_world_export (the thesis has no
 * counterpart; this is a library service).  Some callers cannot call
 * cudaMalloc at the point where they want the state: programs that hand all
 * device memory to their own pool or allocator up front, code that must not
 * hit the device-wide synchronisation a cudaMalloc/cudaFree can cause in
 * the middle of a time-stepped loop, or plugins hosted by a framework that
 * forbids device allocations.  smmo_world_export takes its per-cell scratch
 * with cudaMallocAsync; this entry point takes it from a fixed array inside
 * the library instead and allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine).
 *   - Same arguments and outputs as smmo_world_export; errors (host) is
 *     required.  Synchronises `stream`.
 *   - Limit: at most SMMO_EXPORT_NOALLOC_MAX_CELLS cells in the world
 *     (SMMO_E_UNSUPPORTED above that).  The fixed array (2 MiB + 256 bytes)
 *     is held by every GPU that loads the library until the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: after a cudaDeviceReset of that device (which ends the
 *     context the array lives in) this entry point must not be called
 *     again.
 *   - Every call uses the same array and clears it at its start.  Calls
 *     whose work overlaps on the GPU (other streams, other host threads on
 *     the same device) race on it and must be serialised by the caller. */
#define SMMO_EXPORT_NOALLOC_MAX_CELLS (1u << 24)
int smmo_world_export_noalloc(smmo_world* w, int8_t* kind, int16_t* age,
                              int16_t* energy, uint8_t* state, int64_t* errors,
                              void* stream);
/* total_cells, class ids [Cell, WAgent, Fish, Shark, LAgent, Alive,
 * Candidate] (-1 when absent; class_ids host array of 7), steps done. */
int smmo_world_info(smmo_world* w, int64_t* total_cells, int* class_ids,
                    uint32_t* steps_done);
int smmo_world_destroy(smmo_world* w);

/* ========================================================= street traffic
 * Nagel-Schreckenberg traffic on a street graph (Sec. 7.5): classes Cell
 * {car}, Car {cell, street, v, route, cross}, Source {street}; one step =
 * Car::prepare (accelerate, path, gap against the occupancy at step start,
 * brake with probability p, claim the first cell of the street being
 * entered), Car::move (claim losers stop at the end of their street, cars
 * ending on or passing the last cell of a sink street delete themselves,
 * the rest move), Source::spawn (a producer street with an empty first cell
 * creates a car with v = 0).  The outgoing street at the end of street s in
 * step t is out[s][draw(ROUTE, t, last cell of s) % out_deg[s]]; brake draws
 * are keyed by the car's cell; the lowest cell wins a contested entry. */
typedef struct smmo_traffic smmo_traffic;
/* Registers the classes in a fresh heap and creates cells, cars and
 * producers.  Host arrays of num_streets entries: street_start (cells are
 * numbered street by street, street_start[0] = 0), street_len (>= 2),
 * out_deg (0..3; 0 = sink), out_street (3 per street), is_source.  car_v:
 * device array over all cells, -1 = no car, else the velocity.
 * brake_threshold = floor(p 2^32).  sources_enabled = 0 creates no
 * producers; sinks_enabled = 0 makes sink streets dead ends.  Allocates
 * small street tables with cudaMalloc (freed by smmo_traffic_destroy).
 * Synchronises `stream`. */
int smmo_traffic_create(smmo_heap* heap, int num_streets,
                        const int32_t* street_start, const int32_t* street_len,
                        const int32_t* out_deg, const int32_t* out_street,
                        const uint8_t* is_source, int v_max,
                        uint32_t brake_threshold, int sources_enabled,
                        int sinks_enabled, uint64_t seed, const int8_t* car_v,
                        void* stream, smmo_traffic** out);
/* nsteps steps; asynchronous. */
int smmo_traffic_step(smmo_traffic* w, int nsteps, void* stream);
/* car_v (device, per cell): -1 or the car's velocity; *errors (host,
 * nullable): cells holding two cars + cars whose cell does not point back.
 * Synchronises `stream`. */
int smmo_traffic_export(smmo_traffic* w, int8_t* car_v, int64_t* errors,
                        void* stream);
/* Incoming streets a controller can guard (its inlined inner array). */
#define SMMO_TRAFFIC_MAX_IN 12
/* Adds traffic controllers (Sec. 7.5): ctrl_kind (host, one per street):
 * -1 none, 0 traffic light, 1 smart traffic light, 2 yield controller; a
 * street with fewer than two incoming streets gets none.  phase_len
 * (>= 1): green phase of a light in steps; lookahead (>= 0): cells before
 * the end of an incoming street searched for a waiting car.  Incoming
 * streets are listed in increasing street id (the yield priority); every
 * controller starts green on the first of them, timer 0.  From the next
 * step on, controllers run first and a car from a red street cannot enter
 * the guarded street (speed limit 0 on its first cell).  Once per traffic
 * object; SMMO_E_UNSUPPORTED if a guarded street has more than
 * SMMO_TRAFFIC_MAX_IN incoming streets.  Synchronises `stream`. */
int smmo_traffic_set_controllers(smmo_traffic* w, const int8_t* ctrl_kind, int phase_len,
                                 int lookahead, void* stream);
/* Controller state per street (host arrays of num_streets): index of the
 * green incoming street and phase timer; 0 for unguarded streets.
 * Synchronises `stream`. */
int smmo_traffic_controller_state(smmo_traffic* w, int16_t* green, int16_t* timer, void* stream);
/* num_cells, class ids [Cell, Car, Source, Controller] (host array of 4),
 * steps done; each output nullable. */
int smmo_traffic_info(smmo_traffic* w, int64_t* num_cells, int* class_ids,
                      uint32_t* steps_done);
int smmo_traffic_destroy(smmo_traffic* w);

/* ================================================================ n-body
 * Direct n-body with collision merge (Sec. 7.1, 7.2) and its adjoint.  One
 * class Body {x, y, z, vx, vy, vz, m, id, lx, ly, lz, lvx, lvy, lvz}
 * (the last six: adjoint state).  A step is drift-kick-drift: x += v dt/2,
 * a = G sum_j m_j r_ij / (|r_ij|^2 + eps^2)^{3/2} summed over body ids in
 * increasing order with a fixed FP32 evaluation order (|r|^2 + eps^2 and the
 * sum as fused multiply-adds: s2 = fma(dz, dz, fma(dy, dy, fma(dx, dx,
 * eps^2))), a = fma(m_j / (s2 sqrt(s2)), r, a)) and IEEE division and
 * square root, v += a dt, x += v dt/2; then, if merge != 0, a receiver takes
 * the first lighter body ((m, id) lexicographic) within merge_r in id order,
 * a body picked by several receivers goes to the lowest receiver id, and it
 * merges (v = (v1 m1 + v2 m2)/(m1 + m2), x = midpoint, m = m1 + m2) unless
 * its receiver is itself picked; merged bodies delete themselves. */
typedef struct {
  float G, eps, dt, merge_r;
  int merge;
} smmo_nbody_params;
typedef struct smmo_nbody smmo_nbody;
/* Registers class Body in a fresh heap and creates n bodies with ids
 * 0..n-1.  cols: host array of 7 device pointers (x, y, z, vx, vy, vz, m;
 * n floats each).  Allocates its id-indexed staging arrays with cudaMalloc
 * (freed by smmo_nbody_destroy).  Synchronises `stream`. */
int smmo_nbody_create(smmo_heap* heap, int64_t n, const float* const* cols,
                      const smmo_nbody_params* p, void* stream, smmo_nbody** out);
/* nsteps steps; asynchronous. */
int smmo_nbody_step(smmo_nbody* w, int nsteps, void* stream);
/* out7 (device, 7 x n floats, id-indexed: x, y, z, vx, vy, vz, m), live
 * (device, n bytes), *merges (host, nullable) = merges so far.
 * Synchronises `stream`. */
int smmo_nbody_export(smmo_nbody* w, float* out7, uint8_t* live,
                      int64_t* merges, void* stream);
/* Adjoint of the no-merge run (merge must be 0): runs nsteps steps from the
 * current state keeping (x, v) every ckpt steps, returns the loss
 * L = 1/2 sum m |v|^2 at the end in *loss (host) and initialises the
 * adjoint state (lambda_x = 0, lambda_v = m v).  Synchronises `stream`. */
int smmo_nbody_forward_ckpt(smmo_nbody* w, int nsteps, int ckpt, double* loss,
                            void* stream);
/* Reverse sweep after smmo_nbody_forward_ckpt: every segment is recomputed
 * from its checkpoint, then reversed step by step with the pair kernel
 * g_k = G sum_j H(x_j - x_k)(m_k mu_j - m_j mu_k),
 * H(r) = I/s^3 - 3 r r^T/s^5, mu = dt (lambda_v + dt/2 lambda_x).
 * grad_v0 (device, n x 3 floats, id-indexed) receives dL/dv_0.  The body
 * state afterwards is that of the end of the first segment.  Asynchronous. */
int smmo_nbody_backward(smmo_nbody* w, float* grad_v0, void* stream);
/* Pair terms computed by all force passes so far (live bodies squared per
 * pass: the force sums over the live bodies only) into *pairs (host).
 * Synchronises `stream`. */
int smmo_nbody_pairs(smmo_nbody* w, int64_t* pairs, void* stream);
int smmo_nbody_destroy(smmo_nbody* w);

/* ============================================================ Barnes-Hut
 * 2-D Barnes-Hut with a dynamic quad tree (Sec. 7.3).  Classes NodeBase
 * (abstract) {parent, child_idx, px, py, m}, BodyNode {vx, vy, ax, ay, id},
 * TreeNode {children[4], p1x, p1y, w, frontier, done}; bodies live in the
 * unit square (reflected at its walls).  A step: tree summaries (bottom-up
 * frontier traversal), forces (preorder traversal; a tree node acts as one
 * body when the body is outside its square and w^2 < theta^2 d^2), update,
 * removal of bodies that left their quadrant, reinsertion (compare-and-swap
 * descent, device new of tree nodes), collapse (bottom-up; empty tree nodes
 * deleted, single-body ones replaced by the body).  FP32 in a fixed order,
 * equal to the CPU oracle bit for bit. */
typedef struct {
  float G, eps, dt, theta;  /* eps > 0, theta >= 0 */
} smmo_bh_params;
typedef struct smmo_bh smmo_bh;
/* Registers the classes in a fresh heap (else SMMO_E_FROZEN) and inserts n
 * bodies (body i has id i).  cols: 5 device arrays of n floats: x, y (in
 * [0,1), pairwise distinct), vx, vy, m.  Coincident bodies make device
 * insertion report SMMO_E_BOUNDS (read by smmo_heap_sync).  Synchronises
 * `stream`. */
int smmo_bh_create(smmo_heap* heap, int64_t n, const float* const* cols,
                   const smmo_bh_params* p, void* stream, smmo_bh** out);
/* nsteps steps; asynchronous (no host round trip: each bottom-up traversal
 * is one count of pending children and one do-all whose threads walk up the
 * tree, each node processed by the thread that finishes its last tree-node
 * child).  Capturable in a CUDA graph. */
int smmo_bh_step(smmo_bh* w, int nsteps, void* stream);
/* out5: device, 5 x n floats (x, y, vx, vy, m by id); *tree_nodes (host,
 * nullable) = live TreeNodes.  Synchronises `stream`. */
int smmo_bh_export(smmo_bh* w, float* out5, int64_t* tree_nodes, void* stream);
/* class ids [NodeBase, BodyNode, TreeNode] (host array of 3, nullable) and
 * bottom-up traversals run so far, two per step (nullable). */
int smmo_bh_info(smmo_bh* w, int* class_ids, int64_t* levels);
int smmo_bh_destroy(smmo_bh* w);

/* ================================================================= BFS
 * Frontier-based breadth-first search (Sec. 4.3) over Vertex objects
 * {distance, degree, id, nbr[SMMO_BFS_MAX_DEGREE]} (neighbour handles as an
 * inlined inner array), one parallel_do_and_reduce (OR) per level. */
#define SMMO_BFS_MAX_DEGREE 8
typedef struct smmo_bfs smmo_bfs;
/* Creates n vertices in a fresh heap (else SMMO_E_FROZEN) from a host CSR
 * graph (row_ptr: n + 1 offsets starting at 0, col: neighbour ids);
 * SMMO_E_UNSUPPORTED if a vertex has more than SMMO_BFS_MAX_DEGREE
 * neighbours.  Synchronises `stream`. */
int smmo_bfs_create(smmo_heap* heap, int64_t n, const int32_t* row_ptr,
                    const int32_t* col, void* stream, smmo_bfs** out);
/* Distances from `source`: resets every vertex, then runs up to
 * check_every (1..4096) levels per cooperative launch (a grid barrier
 * between levels; the launch ends after the first level that lowers no
 * distance) and reads the launch's OR results back.  *levels (host,
 * nullable) = largest distance + 1.  Synchronises `stream` once per
 * launch.  A barrier wait that gives up returns SMMO_E_TIMEOUT. */
int smmo_bfs_run(smmo_bfs* w, int32_t source, int check_every, int32_t* levels,
                 void* stream);
/* dist: device array of n int32 (distance by vertex id, 2^31 - 1 =
 * unreachable).  Synchronises `stream`. */
int smmo_bfs_export(smmo_bfs* w, int32_t* dist, void* stream);
int smmo_bfs_destroy(smmo_bfs* w);

/* ============================================================= structure
 * A spring mesh that cracks under load (the finite-element application of
 * Sec. 7.4).  Classes NodeBase (abstract) {x, y, springs[3] (an inlined
 * inner array of Spring handles), num_springs, distance, id}, AnchorNode
 * (fixed), AnchorPullNode {vx, vy} (constant velocity), Node {vx, vy, m},
 * Spring {p1, p2, k, L0, fmax, fx, fy, flag, id}.  One iteration: pull
 * (x += v dt for every AnchorPullNode); `substeps` times
 * Spring::compute_force (d = p2 - p1, F = k (|d| - L0) when |d| > L0 else
 * 0; F > fmax breaks the spring: it leaves both endpoints, a node left
 * without springs is deleted, and it deletes itself; otherwise f = F d/|d|
 * acts on p1 and -f on p2) and Node::update (v = (v + (sum of f in slot
 * order) / m dt)(1 - damping), x += v dt); then the removal of every node
 * that no longer reaches an AnchorNode through springs: a frontier BFS from
 * the AnchorNodes (one parallel_do_and_reduce per level over all node
 * classes in one launch), then the springs of unreached nodes are removed
 * as above.  FP32 in that order, equal to the CPU oracle bit for bit. */
#define SMMO_STRUCT_ANCHOR 0
#define SMMO_STRUCT_PULL 1
#define SMMO_STRUCT_NODE 2
#define SMMO_STRUCT_PHASE_PULL 1
#define SMMO_STRUCT_PHASE_COMPUTE 2
#define SMMO_STRUCT_PHASE_REMOVE 4
typedef struct {
  float dt, damping;
  int32_t substeps;         /* compute steps per iteration (>= 0)      */
  int32_t bfs_check_every;  /* BFS levels per cooperative launch and read-back (1..4096) */
} smmo_structure_params;
typedef struct smmo_structure smmo_structure;
/* Creates the mesh in a fresh heap (else SMMO_E_FROZEN).  Host arrays.
 * Nodes (n): kind (SMMO_STRUCT_*), node_cols = {x, y, vx, vy, m} (vx, vy
 * of anchor nodes and m of non-Node kinds are ignored), slot (3 n spring
 * ids, -1 = empty).  Springs (ns): p1, p2 (node ids), spring_cols = {k,
 * L0, fmax}.  Node i gets id i, spring j id j.  SMMO_E_INVALID_ARG unless
 * every node's slots list exactly the springs that name it.  Synchronises
 * `stream`. */
int smmo_structure_create(smmo_heap* heap, int64_t n, const int8_t* kind,
                          const float* const* node_cols, const int32_t* slot,
                          int64_t ns, const int32_t* p1, const int32_t* p2,
                          const float* const* spring_cols,
                          const smmo_structure_params* p, void* stream,
                          smmo_structure** out);
/* `iterations` iterations of the phases in the bit mask `phases`
 * (SMMO_STRUCT_PHASE_*; 7 = all, in the order pull, compute, remove).  The
 * removal runs up to bfs_check_every BFS levels per cooperative launch (it
 * ends after the first level without frontier) and reads the flags back
 * after each; a barrier wait that gives up returns SMMO_E_TIMEOUT. */
int smmo_structure_step(smmo_structure* w, int iterations, int phases, void* stream);
/* Device output arrays by id (each nullable): nodes (n) node_alive (0/1),
 * x, y, vx, vy (0 for anchors), num_springs, distance (of the last
 * removal; 2^31 - 1 = unreached), slot (3 n spring ids, -1 = empty);
 * springs (ns) spring_alive, fx, fy.  Values of deleted objects are left
 * untouched.  Synchronises `stream`. */
typedef struct {
  uint8_t* node_alive;
  float *x, *y, *vx, *vy;
  int32_t *num_springs, *distance, *slot;
  uint8_t* spring_alive;
  float *fx, *fy;
} smmo_structure_out;
int smmo_structure_export(smmo_structure* w, const smmo_structure_out* out, void* stream);
/* class ids [NodeBase, AnchorNode, AnchorPullNode, Node, Spring] (host, 5,
 * nullable); counters (host, 5, nullable): springs broken, nodes deleted
 * (by breaks and removals), springs removed by the removal phase, BFS
 * levels run, BFS launches (each up to
 * bfs_check_every levels).  Synchronises `stream` if counters. */
int smmo_structure_info(smmo_structure* w, int* class_ids, int64_t* counters, void* stream);
int smmo_structure_destroy(smmo_structure* w);

/* FP32 add/multiply throughput of this GPU: every SM full of threads
 * running eight independent multiply-then-add chains (separate
 * instructions) for `iters` (1..2^20) iterations, timed with CUDA events.
 * *ops_per_s (host) = FP32 operations (one per multiply, one per add) per
 * second, i.e. FP32 instructions per second.  Synchronises `stream`. */
int smmo_measure_fp32_peak(int iters, double* ops_per_s, void* stream);
/* The same with fused multiply-add chains (the peak of the n-body force's
 * roofline, whose fixed evaluation order uses fused multiply-adds):
 * *flops_per_s (host) = floating-point operations per second, two per
 * fused multiply-add.  Synchronises `stream`. */
int smmo_measure_fma_peak(int iters, double* flops_per_s, void* stream);
/* Special-function (reciprocal square root) throughput, measured the same
 * way with eight independent chains of the hardware approximation per
 * thread: *ops_per_s (host) = approximations per second.  The force kernel
 * issues two per pair (square root and reciprocal). */
int smmo_measure_mufu_peak(int iters, double* ops_per_s, void* stream);

/* Self-test of a bounded wait: one CTA waits at the BFS level barrier for a
 * second CTA that never arrives, for `spins` polls of about 100 ns
 * (1..2^20), then records SMMO_E_TIMEOUT (detail 1) in the heap's error
 * word and returns; the
 * caller reads it with smmo_heap_sync.  Synchronises `stream`. */
int smmo_selftest_barrier_timeout(smmo_heap* heap, uint32_t spins, void* stream);

/* Self-test of the branch-free, correctly rounded FP32 square root and
 * reciprocal that the force kernel uses when every coordinate is within
 * 2^18 and eps^2 is in [2^-40, 2^38] (otherwise it uses the IEEE-rounded
 * intrinsics): compares both with __fsqrt_rn / __frcp_rn on every positive
 * float whose bit pattern lies in [lo_bits, hi_bits] (hi_bits < 0x7F800000).
 * out4 (host): mismatches of the square root, of the reciprocal, and the
 * smallest mismatching bit pattern of each (0xFFFFFFFF if none).  The force
 * kernel relies on no mismatch of the square root in [2^-40, 2^40] and of
 * the reciprocal in [2^-60, 2^60].  Allocates 24 bytes with cudaMallocAsync
 * on `stream`; synchronises `stream`. */
int smmo_selftest_fp32_rn(uint32_t lo_bits, uint32_t hi_bits, uint64_t* out4, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SMMO_H */
