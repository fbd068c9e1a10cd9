// heap_internal.h -- host-side heap object shared by the library's .cu files.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "smmo.h"
#include "smmo_core.cuh"

struct ClassInfo {
  std::string name;
  std::vector<smmo_field_desc> fields;   // including inherited (first)
  std::vector<std::string> field_names;  // owned copies of the names
  int parent = -1;
  int abstract = 0;
  std::vector<int> children;
  // geometry (after freeze)
  int ncols = 0;
  int object_bytes = 0;
  smmo::ClassLayout layout{};
};

struct smmo_heap {
  smmo_heap_config cfg{};
  uint8_t* buf = nullptr;
  size_t buf_bytes = 0;
  bool frozen = false;
  int device = 0;
  int num_sms = 0;
  std::vector<ClassInfo> classes;
  smmo::HeapView view{};
  smmo::ClassLayout* d_layouts = nullptr;  // inside buf
  uint32_t* d_scratch = nullptr;           // inside buf: num_blocks + 64 words
  unsigned long long* d_moved = nullptr;   // inside buf: one bit per block (compaction)
  // the last compaction, for smmo_remap_handles: passes run, and the device
  // news and bulk creations counted at its end (-1: no compaction yet)
  uint32_t compact_passes = 0;
  int64_t compact_news = -1, compact_bulks = -1;
  int64_t bulk_calls = 0;                  // bulk_new calls that created objects
  std::vector<smmo_instance_desc> batch;   // instance table (smmo_batch_define)
  smmo::Inst* d_inst = nullptr;            // its device copy, inside buf
};

namespace smmo {
// status helpers
int cuda_status(cudaError_t e);
int freeze(smmo_heap* h, cudaStream_t s);
// concrete classes in the subtree of c (c itself first if concrete)
void concrete_subtree(const smmo_heap* h, int c, std::vector<int>* out);
// enumerate class c into h->view.R, count into st->rcount (asynchronous)
int enumerate(smmo_heap* h, int c, cudaStream_t s);
// A saved enumeration of one class with its own entry buffer and count, so
// that several classes' snapshots can be reused by later do-alls (valid
// while no object of the class is created or deleted).  `view` is the
// heap's view with R and rcnt pointing at the snapshot.
struct Snapshot {
  void* buf = nullptr;  // M entries + the count (device)
  HeapView view{};
  int cls = -1;
  int take(smmo_heap* h, int c, cudaStream_t s);  // (re-)enumerate class c
  // the concrete classes of c's subtree one after the other (for a POLY
  // do-all: each unit takes its class from the block's type id)
  int take_subtree(smmo_heap* h, int c, cudaStream_t s);
  void release();
};
// level l of hierarchical bitmap k (device pointer computed on the host)
inline unsigned long long* bm_level_host(const smmo_heap* h, int k, int l = 0) {
  return h->view.bitmaps + (size_t)k * h->view.bm_words + h->view.level_off[l];
}
// grid for persistent kernels
inline dim3 do_all_grid(const smmo_heap* h) {
  return dim3((unsigned)(h->num_sms * h->cfg.ctas_per_sm));
}

// Method registry: methods are compiled-in do-all kernels.
typedef int (*method_launch_fn)(smmo_heap*, int cls, const void* args, cudaStream_t);
// reducing methods (parallel_do_and_reduce): fold into *out (device)
typedef int (*method_reduce_fn)(smmo_heap*, int cls, const void* args, int op, long long* out, cudaStream_t);
struct MethodEntry {
  const char* name;
  size_t args_size;
  method_launch_fn launch;  // null for reducing methods
  method_reduce_fn reduce;  // null for plain methods
};
const MethodEntry* method_by_id(int id);
}  // namespace smmo

// Per-workload method tables (external linkage: defined in the wl_*.cu files).
extern const smmo::MethodEntry g_methods_test[];
extern const int g_methods_test_n;
extern const smmo::MethodEntry g_methods_wator[];
extern const int g_methods_wator_n;
extern const smmo::MethodEntry g_methods_gol[];
extern const int g_methods_gol_n;
extern const smmo::MethodEntry g_methods_nasch[];
extern const int g_methods_nasch_n;
extern const smmo::MethodEntry g_methods_nbody[];
extern const int g_methods_nbody_n;
extern const smmo::MethodEntry g_methods_bh[];
extern const int g_methods_bh_n;
extern const smmo::MethodEntry g_methods_bfs[];
extern const int g_methods_bfs_n;
extern const smmo::MethodEntry g_methods_structure[];
extern const int g_methods_structure_n;

#ifdef __CUDACC__
// Instantiates the do-all kernel for method M (see smmo_core.cuh).
// The persistent grid holds as many CTAs as can be resident at once
// (occupancy of this instantiation at the configured CTA size, capped by
// ctas_per_sm), so no CTA waits for another to finish before it starts.
template <class M, bool POLY = false>
int launch_do_all_view(smmo_heap* h, int cls, const void* args, cudaStream_t s, const smmo::HeapView* v) {
  const typename M::Args* a = static_cast<const typename M::Args*>(args);
  static int occ_threads = 0, occ_blocks = 0;
  if (occ_threads != h->cfg.threads_per_cta) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, smmo::do_all_kernel<M, POLY>, h->cfg.threads_per_cta, 0) != cudaSuccess || nb < 1) nb = 1;
    occ_blocks = nb;
    occ_threads = h->cfg.threads_per_cta;
  }
  const int per_sm = occ_blocks < h->cfg.ctas_per_sm ? occ_blocks : h->cfg.ctas_per_sm;
  smmo::do_all_kernel<M, POLY><<<h->num_sms * per_sm, h->cfg.threads_per_cta, 0, s>>>(v ? *v : h->view, cls, *a);
  return smmo::cuda_status(cudaGetLastError());
}
template <class M>
int launch_do_all(smmo_heap* h, int cls, const void* args, cudaStream_t s) {
  return launch_do_all_view<M>(h, cls, args, s, nullptr);
}
#define SMMO_METHOD(name, M) {name, sizeof(typename M::Args), &launch_do_all<M>, nullptr}

// Creates the objects that do_all<M> (M::kQueued) left in its queue.
template <class M>
int launch_create_queued(smmo_heap* h, int, const void* args, cudaStream_t s) {
  const typename M::Args* a = static_cast<const typename M::Args*>(args);
  static int occ_threads = 0, occ_blocks = 0;
  if (occ_threads != h->cfg.threads_per_cta) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, smmo::create_queued_kernel<M>, h->cfg.threads_per_cta, 0) !=
            cudaSuccess || nb < 1)
      nb = 1;
    occ_blocks = nb;
    occ_threads = h->cfg.threads_per_cta;
  }
  const int per_sm = occ_blocks < h->cfg.ctas_per_sm ? occ_blocks : h->cfg.ctas_per_sm;
  smmo::create_queued_kernel<M><<<h->num_sms * per_sm, h->cfg.threads_per_cta, 0, s>>>(h->view, *a);
  return smmo::cuda_status(cudaGetLastError());
}

template <class M, bool POLY = false>
int launch_do_all_reduce_view(smmo_heap* h, int cls, const void* args, int op, long long* out, cudaStream_t s,
                              const smmo::HeapView* v) {
  const typename M::Args* a = static_cast<const typename M::Args*>(args);
  static int occ_threads = 0, occ_blocks = 0;
  if (occ_threads != h->cfg.threads_per_cta) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, smmo::do_all_reduce_kernel<M, POLY>, h->cfg.threads_per_cta, 0) !=
            cudaSuccess || nb < 1)
      nb = 1;
    occ_blocks = nb;
    occ_threads = h->cfg.threads_per_cta;
  }
  const int per_sm = occ_blocks < h->cfg.ctas_per_sm ? occ_blocks : h->cfg.ctas_per_sm;
  smmo::do_all_reduce_kernel<M, POLY><<<h->num_sms * per_sm, h->cfg.threads_per_cta, 0, s>>>(v ? *v : h->view, cls, *a, op, out);
  return smmo::cuda_status(cudaGetLastError());
}
template <class M>
int launch_do_all_reduce(smmo_heap* h, int cls, const void* args, int op, long long* out, cudaStream_t s) {
  return launch_do_all_reduce_view<M>(h, cls, args, op, out, s, nullptr);
}
#define SMMO_METHOD_REDUCE(name, M) {name, sizeof(typename M::Args), nullptr, &launch_do_all_reduce<M>}
#endif
