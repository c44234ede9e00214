// D2Q9 instantiations of the step, set-up and read-back kernels.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q9(int nc, int precision, int collision) { return ops_for<9>(nc, precision, collision); }
}  // namespace lbm
