// D3Q19 instantiations of the step, set-up and read-back kernels.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q19(int nc, int precision, int collision) { return ops_for<19>(nc, precision, collision); }
}  // namespace lbm
