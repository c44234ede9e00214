// Host helpers shared by the single-lattice and the batched C ABI. Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "lbm.h"
#include "lbm_core.cuh"
#include "lbm_ops.h"

namespace lbm {

// Validates one lattice description and fills its kernel parameters and dispatch table.
lbm_status make_params(const lbm_grid* grid, int nc, const lbm_component* comps, const lbm_eos* eos, double tau,
                       Params* out, const Ops** ops_out, std::string* why);

// Diagnostics of a state given as device arrays of component densities (nc * N) and EOS
// pressures (N); work: device buffer of at least 12 N + 256 bytes (lbm_diag.cu).
lbm_status diagnostics(const Params& P, int nc, int D, const lbm_diag_params* dp, const double* rho,
                       const double* p, void* work, cudaStream_t s, lbm_diag_result* out, std::string* why);

}  // namespace lbm
