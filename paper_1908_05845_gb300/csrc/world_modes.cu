// world_modes.cu -- the Wa-Tor step kernels other than the four plain
// do-alls of world.cu (smmo_world_set_step_kernels): creations queued for a
// launch of their own, and updates that run only on the agents their
// prepare marked; the fused phases are in world_phased.cu.  Every mode
// computes what the four do-alls compute.  Translation units of their own,
// so that these kernel instantiations compile in parallel with world.cu.
#include "world_wator.cuh"

namespace {

// The same methods with their creations queued (smmo_core.cuh, DeferQueue)
// and made by a separate launch after the update.
struct FishUpdateQ : FishUpdate {
  static constexpr bool kQueued = true;
  __device__ static DeferQueue queue(const Args& a) { return a.fq; }
};
struct SharkUpdateQ : SharkUpdate {
  static constexpr bool kQueued = true;
  __device__ static DeferQueue queue(const Args& a) { return a.sq; }
};
// Marking prepares and filtered updates (smmo_core.cuh): the update runs
// only on the agents whose prepare posted a request (or starved); the rest
// would return at once.
struct FishPrepareM : FishPrepare { static constexpr bool kMarks = true; };
struct SharkPrepareM : SharkPrepare { static constexpr bool kMarks = true; };
struct FishUpdateF : FishUpdate { static constexpr bool kFiltered = true; };
struct SharkUpdateF : SharkUpdate { static constexpr bool kFiltered = true; };
struct FishUpdateQF : FishUpdateQ { static constexpr bool kFiltered = true; };
struct SharkUpdateQF : SharkUpdateQ { static constexpr bool kFiltered = true; };
}  // namespace

smmo::method_launch_fn wator_mode_launcher(int which, int mode) {
  if ((mode & 3) != SMMO_WATOR_FOUR_DO_ALLS) return wator_phased_launcher(which, mode);
  const bool q = (mode & SMMO_WATOR_QUEUED_CREATION) != 0, mk = (mode & SMMO_WATOR_MARKED_UPDATE) != 0;
  switch (which) {
    case kWFishPrepare: return mk ? &launch_do_all<FishPrepareM> : nullptr;
    case kWSharkPrepare: return mk ? &launch_do_all<SharkPrepareM> : nullptr;
    case kWFishUpdate:
      return q ? (mk ? &launch_do_all<FishUpdateQF> : &launch_do_all<FishUpdateQ>)
               : (mk ? &launch_do_all<FishUpdateF> : nullptr);
    case kWSharkUpdate:
      return q ? (mk ? &launch_do_all<SharkUpdateQF> : &launch_do_all<SharkUpdateQ>)
               : (mk ? &launch_do_all<SharkUpdateF> : nullptr);
    case kWFishCreate: return q ? &launch_create_queued<FishUpdateQ> : nullptr;
    case kWSharkCreate: return q ? &launch_create_queued<SharkUpdateQ> : nullptr;
    default: return nullptr;
  }
}
