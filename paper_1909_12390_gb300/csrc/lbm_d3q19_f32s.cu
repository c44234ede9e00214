// D3Q19 instantiations with FP32-shifted storage: step, set-up and read-back kernels.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q19_f32s(int nc, int collision) {
  return collision ? ops_nc<19, PrecF32S, 1>(nc) : ops_nc<19, PrecF32S, 0>(nc);
}
}  // namespace lbm
