// D2Q9, FP32-shifted storage, MRT collision: step, set-up and read-back kernels for 1..4 components.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q9_f32s_mrt(int nc) { return ops_nc<9, PrecF32S, 1>(nc); }
}  // namespace lbm
