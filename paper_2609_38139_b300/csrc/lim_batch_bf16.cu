// lim_batch_bf16.cu -- batch kernels with bf16 message storage.
#include "lim_batch.cuh"

namespace lim {

const void *batch_fn_bf16(int warp, int rule, int fb) {
  using namespace batch_detail;
  return warp ? pick_kernel<TeamWarp, LIM_PREC_BF16>(rule, fb) : pick_kernel<TeamCTA, LIM_PREC_BF16>(rule, fb);
}

}  // namespace lim
