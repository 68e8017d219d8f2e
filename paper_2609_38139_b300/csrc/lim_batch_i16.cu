// lim_batch_i16.cu -- batch kernels with i16 message storage.
#include "lim_batch.cuh"

namespace lim {

const void *batch_fn_i16(int warp, int rule, int fb) {
  using namespace batch_detail;
  return warp ? pick_kernel<TeamWarp, LIM_PREC_I16>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_I16>(rule, fb);
}

}  // namespace lim
