// lim_batch_bf16.cu -- batch kernels with bf16 message storage.
#include "lim_batch.cuh"
#include "lim_lane.cuh"

namespace lim {

const void *batch_fn_bf16(int kind, int rule, int fb) {
  using namespace batch_detail;
  if (kind == kKindLane) return fb == LIM_FB_CHECK_MOVE ? lane_detail::pick_lane_kernel<LIM_PREC_BF16>(rule) : nullptr;
  return kind == kKindWarp ? pick_kernel<TeamWarp, LIM_PREC_BF16>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_BF16>(rule, fb);
}

}  // namespace lim
