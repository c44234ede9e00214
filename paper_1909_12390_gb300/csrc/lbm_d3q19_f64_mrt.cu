// D3Q19, FP64 storage, MRT collision: step, set-up and read-back kernels for 1..4 components.
#include "lbm_kernels.cuh"

namespace lbm {
const Ops* ops_q19_f64_mrt(int nc) { return ops_nc<19, PrecF64, 1>(nc); }
}  // namespace lbm
