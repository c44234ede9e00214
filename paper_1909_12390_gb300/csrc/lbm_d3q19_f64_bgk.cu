// D3Q19, FP64 storage, BGK collision: step, set-up and read-back kernels for 1..4 components.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q19_f64_bgk(int nc) { return ops_nc<19, PrecF64, 0>(nc); }
}  // namespace lbm
