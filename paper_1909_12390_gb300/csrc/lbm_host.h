// Host helpers shared by the single-lattice and the batched C ABI. Internal to the library.
#pragma once

#include <string>

#include "lbm.h"
#include "lbm_core.cuh"
#include "lbm_ops.h"

namespace lbm {

// Validates one lattice description and fills its kernel parameters and dispatch table.
lbm_status make_params(const lbm_grid* grid, int nc, const lbm_component* comps, const lbm_eos* eos, double tau,
                       Params* out, const Ops** ops_out, std::string* why);

}  // namespace lbm
