// D2Q9, FP32-shifted storage, BGK collision: step, set-up and read-back kernels for 1..4 components.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q9_f32s_bgk(int nc) { return ops_nc<9, PrecF32S, 0>(nc); }
}  // namespace lbm
