// lim_batch_f32.cu -- batch kernels with f32 message storage.
#include "lim_batch.cuh"
#include "lim_lane.cuh"

namespace lim {

const void *batch_fn_f32(int kind, int rule, int fb) {
  using namespace batch_detail;
  if (kind == kKindLane) return fb == LIM_FB_CHECK_MOVE ? lane_detail::pick_lane_kernel<LIM_PREC_F32>(rule) : nullptr;
  return kind == kKindWarp ? pick_kernel<TeamWarp, LIM_PREC_F32>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_F32>(rule, fb);
}

// The plain baseline path exists for binary32 messages only.
void plain_fns_f32(int rule, int fb, const void **init, const void **tick, const void **finish) {
  batch_detail::pick_plain<LIM_PREC_F32>(rule, fb, init, tick, finish);
}

}  // namespace lim
