// wl_test.cu -- small methods used by the allocator and enumeration tests
// and by the allocation microbenchmark (the thesis' Linux-scalability
// experiment, Sec. 5.6.4: many threads allocate objects, then free them).
#include "heap_internal.h"
#include "levels.cuh"
#include "smmo_core.cuh"

using namespace smmo;

namespace {

// field[col] += value  (int32 column)
struct AddI32 {
  struct Args { uint32_t col; int32_t value; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    int32_t* f = field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col]), self);
    *f += a.value;
  }
};

// Each visited object allocates `k` objects of class `target` and writes
// `marker` into their int32 column `col` and its own value of column
// `src_col` into column `col2` (so the test can check who allocated what).
struct AllocK {
  struct Args { uint32_t target; uint32_t k; uint32_t col; uint32_t col2; uint32_t src_col; int32_t marker; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t mine = *field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.src_col]), self);
    for (uint32_t i = 0; i < a.k; ++i) {
      const uint32_t o = smmo_new(h, a.target);
      if (o == kNull) return;
      *field_ptr<int32_t>(h, __ldg(&h.cls[a.target].col_off[a.col]), o) = a.marker;
      *field_ptr<int32_t>(h, __ldg(&h.cls[a.target].col_off[a.col2]), o) = mine;
    }
  }
};

// Deletes itself when (column col) % mod == rem.
struct FreeSelfIf {
  struct Args { uint32_t col; int32_t mod; int32_t rem; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t v = *field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col]), self);
    const int32_t m = a.mod > 0 ? ((v % a.mod) + a.mod) % a.mod : 0;
    if (a.mod <= 0 || m == a.rem) smmo_delete(h, self);
  }
};

// Deletes the object referenced by HANDLE column `col` (an object of
// another class) and clears the reference.
struct FreeRef {
  struct Args { uint32_t col; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    uint32_t* r = field_ptr<uint32_t>(h, __ldg(&h.cls[c].col_off[a.col]), self);
    if (*r != kNull) { smmo_delete(h, *r); *r = kNull; }
  }
};

// Replaces itself by a new object of class `target` carrying column col.
struct Replace {
  struct Args { uint32_t target; uint32_t col; uint32_t tcol; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t v = *field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col]), self);
    const uint32_t o = smmo_new(h, a.target);
    if (o != kNull) *field_ptr<int32_t>(h, __ldg(&h.cls[a.target].col_off[a.tcol]), o) = v;
    smmo_delete(h, self);
  }
};

// HANDLE column col_ref = table[int32 column col_idx] (wiring references
// between classes after both were created).
struct SetRefFrom {
  struct Args { uint32_t col_ref; uint32_t col_idx; const uint32_t* table; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const int32_t i = *field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col_idx]), self);
    *field_ptr<uint32_t>(h, __ldg(&h.cls[c].col_off[a.col_ref]), self) = a.table[i];
  }
};

// Reducing method: the value of int32 column col (or 1 if count is set).
struct ValueI32 {
  struct Args { uint32_t col; uint32_t count; };
  __device__ static long long run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    if (a.count) return 1;
    return *field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col]), self);
  }
};

// Batch method: an object of a class with a SMMO_INSTANCE field updates its
// int32 column col from the row of its instance, v = v * param[0] +
// param[1] + kind (64-bit arithmetic, low 32 bits kept), and adds the
// instance's id to column col_id (one launch over every instance).
struct BatchAffine {
  struct Args { uint32_t col; uint32_t col_id; };
  __device__ static void run(const HeapView& h, const Args& a, uint32_t c, uint32_t self) {
    const Inst* in = instance_of(h, c, self);
    if (!in) { set_error(h, SMMO_E_BOUNDS, self); return; }
    int32_t* v = field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col]), self);
    const long long r = (long long)*v * __ldg(&in->param[0]) + __ldg(&in->param[1]) + __ldg(&in->kind);
    *v = (int32_t)(uint32_t)(unsigned long long)r;
    int32_t* idc = field_ptr<int32_t>(h, __ldg(&h.cls[c].col_off[a.col_id]), self);
    *idc += (int32_t)__ldg(&in->id);
  }
};

}  // namespace

const smmo::MethodEntry g_methods_test[] = {
    SMMO_METHOD("test.add_i32", AddI32),
    SMMO_METHOD("test.alloc_k", AllocK),
    SMMO_METHOD("test.free_self_if", FreeSelfIf),
    SMMO_METHOD("test.free_ref", FreeRef),
    SMMO_METHOD("test.replace", Replace),
    SMMO_METHOD("test.set_ref_from", SetRefFrom),
    SMMO_METHOD_REDUCE("test.value_i32", ValueI32),
    SMMO_METHOD("test.batch_affine", BatchAffine),
};
const int g_methods_test_n = sizeof(g_methods_test) / sizeof(g_methods_test[0]);

// ------------------------------------------------ bounded barrier self-test
namespace {
// One CTA waits at a level barrier that expects two CTAs: its own arrival
// is the only one, so nothing releases it and the wait runs out after
// `spins` polls, recording SMMO_E_TIMEOUT (detail 1, the first level).
__global__ void k_barrier_nobody_comes(HeapView h, unsigned long long* ctl, unsigned spins) {
  int any = 0;
  smmo::level_barrier(h, ctl, 0u, false, 2u, &any, spins);
}
}  // namespace

extern "C" int smmo_selftest_barrier_timeout(smmo_heap* h, uint32_t spins, void* stream) {
  if (!h || !h->frozen || spins < 1 || spins > (1u << 20)) return SMMO_E_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* arrive = nullptr;
  cudaError_t e = cudaMallocAsync(&arrive, sizeof(unsigned long long) * smmo::kBarrierWords, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(arrive, 0, sizeof(unsigned long long) * smmo::kBarrierWords, s);
  if (e == cudaSuccess) {
    k_barrier_nobody_comes<<<1, 64, 0, s>>>(h->view, arrive, spins);
    e = cudaGetLastError();
  }
  if (arrive) cudaFreeAsync(arrive, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? SMMO_OK : smmo::cuda_status(e);
}
