// lim_batch_i16.cu -- batch kernels with i16 message storage.
#include "lim_batch.cuh"
#include "lim_lane.cuh"

namespace lim {

const void *batch_fn_i16(int kind, int rule, int fb) {
  using namespace batch_detail;
  if (kind == kKindLane) return fb == LIM_FB_CHECK_MOVE ? lane_detail::pick_lane_kernel<LIM_PREC_I16>(rule) : nullptr;
  return kind == kKindWarp ? pick_kernel<TeamWarp, LIM_PREC_I16>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_I16>(rule, fb);
}

}  // namespace lim
