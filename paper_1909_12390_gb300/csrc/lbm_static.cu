// lbm_step_static: the two-kernel step on populations the caller keeps in its own device
// memory, with every scratch buffer in one fixed device array of this file, so the call
// allocates nothing. See include/lbm.h for who needs this and its limits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_kernels.cuh"

namespace {

// Scratch layout: [0, 256) status word and step counter, then the pseudo-potential of up to
// LBM_STATIC_MAX_SITES sites in FP64 (FP32 storage uses the first half).
constexpr size_t kHeader = 256;
constexpr size_t kScratchBytes = kHeader + (size_t)LBM_STATIC_MAX_SITES * sizeof(double);

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

__global__ void k_static_reset(int* status, long long* t, long long t0) {
  *status = 0;
  *t = t0;
}

thread_local char g_msg[256];

lbm_status say(lbm_status st, const char* what, const char* detail = "") {
  snprintf(g_msg, sizeof g_msg, "%s%s", what, detail);
  return st;
}

}  // namespace

extern "C" {

lbm_status lbm_step_static(const lbm_grid* grid, int nc, const lbm_component* comps, const lbm_eos* eos,
                           double tau, void* f_device, int64_t t0, int64_t n, void* stream, int64_t* t_out) {
  g_msg[0] = 0;
  if (!f_device) return say(LBM_ERR_ARG, "f_device is NULL");
  if (n < 0 || t0 < 0) return say(LBM_ERR_ARG, "n and t0 must be >= 0");
  lbm::Params P{};
  const lbm::Ops* ops = nullptr;
  std::string why;
  lbm_status st = lbm::make_params(grid, nc, comps, eos, tau, &P, &ops, &why);
  if (st != LBM_OK) return say(st, why.c_str());
  if (P.N > (int64_t)LBM_STATIC_MAX_SITES)
    return say(LBM_ERR_ARG, "grid has more sites than LBM_STATIC_MAX_SITES");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return say(LBM_ERR_CUDA, "cudaGetDevice: ", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return say(LBM_ERR_CUDA, "device ordinal out of range");
  unsigned char* base = nullptr;
  {
    // first call on this device: the symbol's device address, with this device current
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) return say(LBM_ERR_CUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
      g_scratch_ptr[dev] = (unsigned char*)p;
    }
    base = g_scratch_ptr[dev];
  }
  int* status = (int*)base;
  long long* t_dev = (long long*)(base + 64);
  void* psi = base + kHeader;
  cudaStream_t s = (cudaStream_t)stream;

  k_static_reset<<<1, 1, 0, s>>>(status, t_dev, (long long)t0);
  for (int64_t i = 0; i < n; ++i) {
    const int parity = (int)((t0 + i) & 1);
    ops->psi(P, f_device, psi, status, parity, s);
    ops->collide(P, f_device, psi, status, t_dev, parity, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return say(LBM_ERR_CUDA, "launch: ", cudaGetErrorString(e));
  int hs = 0;
  long long ht = 0;
  e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&ht, t_dev, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return say(LBM_ERR_CUDA, "sync: ", cudaGetErrorString(e));
  if (t_out) *t_out = ht;
  if (hs & lbm::ST_NONFINITE) return say(LBM_ERR_NONFINITE, "non-finite density or psi^2");
  if (hs & lbm::ST_PSI_DOMAIN) return say(LBM_ERR_PSI_DOMAIN, "psi^2 < 0 or b_m n >= 1");
  // any other status bit (none of the two-kernel step's kernels raises one today) is reported
  // as the context path reports it, never as success
  if (hs) return say(LBM_ERR_TIMEOUT, "device status bits set");
  return LBM_OK;
}

const char* lbm_step_static_error(void) { return g_msg; }

}  // extern "C"
