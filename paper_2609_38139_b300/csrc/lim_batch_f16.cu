// lim_batch_f16.cu -- batch kernels with f16 message storage.
#include "lim_batch.cuh"

namespace lim {

const void *batch_fn_f16(int warp, int rule, int fb) {
  using namespace batch_detail;
  return warp ? pick_kernel<TeamWarp, LIM_PREC_F16>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_F16>(rule, fb);
}

}  // namespace lim
