// D2Q9 instantiations with FP64 storage: step, set-up and read-back kernels.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q9_f64(int nc, int collision) {
  return collision ? ops_nc<9, PrecF64, 1>(nc) : ops_nc<9, PrecF64, 0>(nc);
}
}  // namespace lbm
