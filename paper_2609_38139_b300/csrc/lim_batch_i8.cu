// lim_batch_i8.cu -- batch kernels with i8 message storage.
#include "lim_batch.cuh"

namespace lim {

const void *batch_fn_i8(int warp, int rule, int fb) {
  using namespace batch_detail;
  return warp ? pick_kernel<TeamWarp, LIM_PREC_I8>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_I8>(rule, fb);
}

}  // namespace lim
