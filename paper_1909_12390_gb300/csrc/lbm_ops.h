// Dispatch table between the host context (lbm_capi.cu) and the kernel instantiations of one
// lattice (lbm_d2q9.cu, lbm_d3q19.cu). Internal to the library.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct Params;
struct FusedArgs;

struct Ops {
  void (*psi)(const Params&, const void* f, void* psi, int* status, int parity, cudaStream_t);
  void (*collide)(const Params&, void* f, const void* psi, const int* status, long long* t_dev, int parity,
                  cudaStream_t);
  cudaError_t (*fused)(const Params&, void* f, void* psi, int* status, long long* t_dev, const FusedArgs&,
                       cudaStream_t);
  int (*fused_max_blocks)();  // co-resident blocks of the fused kernel on this device
  // plane-range fused step (D3Q19 only; cudaErrorNotSupported / 0 otherwise)
  cudaError_t (*fused3)(const Params&, void* f, int* status, long long* t_dev, const FusedArgs&, cudaStream_t);
  int (*fused3_max_blocks)(int smem_bytes);
  void (*init)(const Params&, void* f, const double* rho, const double* u, cudaStream_t);
  void (*get_f)(const Params&, const void* f, double* out, int parity, cudaStream_t);
  void (*set_f)(const Params&, void* f, const double* in, cudaStream_t);
  void (*fields)(const Params&, const void* f, const void* psi, double* rho, double* u, double* p,
                 double* psi_out, int parity, cudaStream_t);
  void (*mass)(const Params&, const void* f, double* partial, double* out, cudaStream_t);
  int store_bytes;  // bytes per stored population
  int psi_bytes;    // bytes per stored pseudo-potential value
  int arith_bytes;  // bytes of the arithmetic type (moments kept by k_fused3)
  int fused_tx;     // fused-kernel tile: sites along x
  int fused_ty;     // and along y (1 for D2Q9)
  int fused_group;  // planes per synchronisation round
  int fused3_wpc;   // plane-range kernel: workers per CTA
  int fused3_flags; // and progress counters per worker
  // the collide pass reading the state in fin and writing the next one to fout
  void (*collide_oop)(const Params&, const void* fin, void* fout, const void* psi, const int* status,
                      long long* t_dev, int parity, cudaStream_t);
  // trailing fused step (D3Q19 only; cudaErrorNotSupported / 0 otherwise): psi of the step
  // from A.psi_ring[t & 1], psi of the next step into A.psi_ring[(t + 1) & 1]
  cudaError_t (*trail3)(const Params&, void* f, int* status, long long* t_dev, const FusedArgs&, cudaStream_t);
  int (*trail3_max_blocks)();  // co-resident CTAs of the trailing step on this device
  // task-queue one-pass step (D3Q19 only; cudaErrorNotSupported / 0 otherwise), psi fields as
  // for trail3
  cudaError_t (*trailq)(const Params&, void* f, int* status, long long* t_dev, const FusedArgs&, cudaStream_t);
  int (*trailq_max_blocks)();  // resident CTAs of the task-queue step on this device
  int trailq_chunk;            // sites per task
  int trailq_lag;              // planes between a collision and the psi task placed after it
};

// one translation unit per lattice, storage type and collision
const Ops* ops_q9_f64_bgk(int nc);
const Ops* ops_q9_f64_mrt(int nc);
const Ops* ops_q9_f32s_bgk(int nc);
const Ops* ops_q9_f32s_mrt(int nc);
const Ops* ops_q19_f64_bgk(int nc);
const Ops* ops_q19_f64_mrt(int nc);
const Ops* ops_q19_f32s_bgk(int nc);
const Ops* ops_q19_f32s_mrt(int nc);

inline const Ops* ops_get(int Q, int fp32, int mrt, int nc) {
  if (Q == 9) {
    if (fp32) return mrt ? ops_q9_f32s_mrt(nc) : ops_q9_f32s_bgk(nc);
    return mrt ? ops_q9_f64_mrt(nc) : ops_q9_f64_bgk(nc);
  }
  if (fp32) return mrt ? ops_q19_f32s_mrt(nc) : ops_q19_f32s_bgk(nc);
  return mrt ? ops_q19_f64_mrt(nc) : ops_q19_f64_bgk(nc);
}

}  // namespace lbm
