// Host side of the C ABI declared in include/lbm.h: argument validation, the Peng-Robinson
// component parameters of Section 3.2, device allocation, the step loop (replayed from a
// captured CUDA graph once it is long enough) and read-back.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_core.cuh"
#include "lbm_host.h"
#include "lbm_kernels.cuh"
#include "lbm_ops.h"

namespace lbm {

__global__ void k_mass_final(const double* partial, int nblocks, int nc, MassShift shift, double* out) {
  __shared__ double sh[256];
  for (int c = 0; c < nc; ++c) {
    double v = 0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * nc + c];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sh[0] + shift.v[c];
    __syncthreads();
  }
}

}  // namespace lbm

namespace {

const double kOmegaA = 0.45724;
const double kOmegaB = 0.0778;
const int kGraphSteps = 64;  // steps per captured graph (even, so parity is fixed)

thread_local std::string g_create_error;

}  // namespace

struct lbm_ctx {
  lbm_grid grid{};
  int nc = 0, Q = 0, precision = 0, collision = 0;
  lbm::Params P{};
  const lbm::Ops* ops = nullptr;
  bool ref_given = false;
  void* f = nullptr;
  void* psi = nullptr;
  int* status = nullptr;
  long long* t_dev = nullptr;
  double* partial = nullptr;
  double* mass_dev = nullptr;
  double* scratch = nullptr;  // fields and staging, (nc + 5) * N doubles, allocated on demand
  cudaStream_t own = nullptr, stream = nullptr;
  int64_t t = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  // step path: the fused kernel when its tiling fits the grid and its blocks are co-resident
  int path_request = LBM_PATH_AUTO;
  bool fused = false;
  // trailing step: the step whose psi fargs.psi_ring[t & 1] holds, -1 when stale (any change of
  // the state other than a trailing step makes it stale)
  int64_t trail_t = -1;
  lbm::FusedArgs fargs{};
  cudaError_t launch_err = cudaSuccess;
  // per-kernel event timing (lbm_profile): events recorded around every launch on the stream
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_marks[3];  // (start, stop) pool indices per kernel kind
  size_t ev_used = 0;
  // adjoint recording (lbm_record): checkpoints of the raw storage every ck_every steps
  std::vector<void*> ckpt;  // pointers into ckpt_base, one per segment
  void* ckpt_base = nullptr;
  size_t ckpt_bytes = 0;
  // captured step sequences of lbm_record's segments, by (steps, parity of the first step)
  std::vector<std::pair<std::pair<int64_t, int>, cudaGraphExec_t>> seg_graphs;
  int ck_every = 0;
  int adj_snaps = 0;  // lbm_adjoint: state slots per segment (0: every state of a segment)
  bool adj_overlap = true;  // lbm_adjoint: replay beside the reverse sweep when memory allows
  int64_t rec_t0 = -1, rec_n = 0;
  std::string err;
};

namespace lbm {
struct AdjFns {
  void (*seed)(const Params&, const double*, void* X, void* rbB, cudaStream_t);
  void (*pass_a)(const Params&, const void* f, const void* psi, const void* X, const void* rbB, void* X_out,
                 void* Fb, void* rho, int parity, double* gpart, cudaStream_t);
  void (*pass_b)(const Params&, const void* psi, const void* Fb, const void* rho, void* rbB, double* kpart,
                 cudaStream_t);
  // pass B of lam(t + 1) (psi_t1, F_in, rho_in) then pass A of step t (f, psi_t, X -> X_out,
  // F_out, rho_out): one fused launch for D2Q9, the two passes for D3Q19 (through rbB)
  void (*pass_ab)(const Params&, const void* f, const void* psi_t, const void* psi_t1, const void* X, void* X_out,
                  const void* F_in, void* F_out, const void* rho_in, void* rho_out, void* rbB, int parity,
                  double* gpart, double* kpart, cudaStream_t);
  void (*init_grad)(const Params&, const void* X, const void* rbB, double* drho0, cudaStream_t);
  unsigned (*rows)(const Params&);  // rows of the partial-sum arrays (one per block of any pass)
  int real_bytes;
};
const AdjFns* adj_fns(int Q, int nc, int precision, int mrt);
}  // namespace lbm

namespace {

lbm_status fail(lbm_ctx* c, lbm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c)
    c->err = buf;
  else
    g_create_error = buf;
  return st;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  // a failed call leaves the runtime's last error set: clear it, so that a later call (of this
  // or another context) does not report it as its own
  cudaGetLastError();
  return fail(c, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

// Host <-> device copies of caller arrays. A host range that straddles a page-locked registration
// (part registered, part not) is refused by the copy itself with cudaErrorInvalidValue; such a
// range goes through a pageable bounce buffer instead (the call synchronises the stream then).
cudaError_t copy_in(void* dst, const void* src, size_t n, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s);
  if (e != cudaErrorInvalidValue) return e;
  cudaGetLastError();
  std::vector<char> tmp((const char*)src, (const char*)src + n);
  e = cudaMemcpyAsync(dst, tmp.data(), n, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}
cudaError_t copy_out(void* dst, const void* src, size_t n, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s);
  if (e != cudaErrorInvalidValue) return e;
  cudaGetLastError();
  std::vector<char> tmp(n);
  e = cudaMemcpyAsync(tmp.data(), src, n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) std::memcpy(dst, tmp.data(), n);
  return e;
}

#define CK(ctx, call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

double m_factor(double w) {
  return w <= 0.49 ? 0.374640 + 1.54226 * w - 0.26992 * w * w
                   : 0.379642 + 1.48503 * w - 0.164423 * w * w + 0.016666 * w * w * w;
}

int rows_q(int Q, int i) { return Q == 9 ? lbm::Lat<9>::krow(i) : lbm::Lat<19>::krow(i); }
int nk_q(int Q) { return Q == 9 ? lbm::Lat<9>::NK : lbm::Lat<19>::NK; }
int norm_q(int Q, int k) { return Q == 9 ? lbm::mnorm<9>(k) : lbm::mnorm<19>(k); }

lbm_status ensure_scratch(lbm_ctx* c) {
  if (c->scratch) return LBM_OK;
  size_t n = (size_t)(c->nc + 5) * (size_t)c->P.N + 8;  // fields, then 8 words for k_check_init
  CK(c, cudaMalloc(&c->scratch, n * sizeof(double)));
  return LBM_OK;
}

// Validation of lbm_init's inputs on the device (they are copied there anyway): out[s] =
// smallest density of component s as its bit pattern (positive doubles order like their bits),
// out[4] = smallest flat index of a density that is not finite and > 0, out[5] = 1 if some u
// is not finite. out[0..4] start at all ones, out[5] at 0.
__global__ void k_check_init(const double* __restrict__ rho, const double* __restrict__ u, long long N, int nc,
                             unsigned long long* out) {
  unsigned long long lo[4] = {~0ull, ~0ull, ~0ull, ~0ull};
  unsigned long long bad = ~0ull;
  bool ubad = false;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)nc * N; i += stride) {
    const double v = rho[i];
    if (!(v > 0) || !isfinite(v)) {
      bad = min(bad, (unsigned long long)i);
    } else {
      const int s = (int)(i / N);
      const unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (k == s) lo[k] = min(lo[k], b);
    }
  }
  if (u)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * N; i += stride)
      ubad = ubad || !isfinite(u[i]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long x = lo[k];
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0 && k < nc && x != ~0ull) atomicMin(&out[k], x);
  }
  for (int o = 16; o > 0; o >>= 1) bad = min(bad, __shfl_xor_sync(0xffffffffu, bad, o));
  if ((threadIdx.x & 31) == 0 && bad != ~0ull) atomicMin(&out[4], bad);
  if (__any_sync(0xffffffffu, ubad) && (threadIdx.x & 31) == 0) atomicExch(&out[5], 1ull);
}

// Allocation range [start, start + size) that the driver records for address p: the
// cudaHostAlloc / cudaHostRegister range for page-locked host memory, the allocation for device
// memory. The driver entry point is looked up through the runtime, so the library links no
// driver library of its own. False when the driver knows no range for p.
bool pointer_range(const void* p, uintptr_t* start, size_t* size) {
  using Fn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static Fn fn = []() -> Fn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return (Fn)f;
  }();
  if (!fn) return false;
  CUdeviceptr s0 = 0;
  size_t n0 = 0;
  if (fn(&s0, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)p) != CUDA_SUCCESS ||
      fn(&n0, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)p) != CUDA_SUCCESS)
    return false;
  *start = (uintptr_t)s0;
  *size = n0;
  return true;
}

// Device address of the host range [p, p + n): non-null only when the whole range lies inside
// one page-locked allocation mapped into the device's address space (cudaHostAlloc,
// cudaHostRegister). The kernels then read or write the caller's buffer directly over the
// host link, which on a Grace-Blackwell node is several times faster than a copy-engine
// transfer of the same bytes; any other host memory (including a range that runs past its
// registration into unregistered memory, or across two registrations) is staged through
// device memory by the caller.
template <class T>
T* mapped_range(T* p, size_t n) {
  if (!p || n == 0) return nullptr;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
  uintptr_t start = 0;
  size_t size = 0;
  const uintptr_t a = (uintptr_t)p;
  if (!pointer_range(p, &start, &size) || a < start || n > (start + size - a) / sizeof(T)) return nullptr;
  return (T*)at.devicePointer;
}

lbm_status sync_status(lbm_ctx* c) {
  int st = 0;
  long long t = 0;
  CK(c, cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(&t, c->t_dev, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  CK(c, cudaGetLastError());
  c->t = t;
  if (st == 0) return LBM_OK;
  CK(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (st & lbm::ST_NONFINITE) return fail(c, LBM_ERR_NONFINITE, "non-finite density or psi^2 at step %lld", t);
  if (st & lbm::ST_PSI_DOMAIN)
    return fail(c, LBM_ERR_PSI_DOMAIN, "psi^2 < 0 or b_m n >= 1 at step %lld", t);
  return fail(c, LBM_ERR_TIMEOUT, "device wait timed out at step %lld", t);
}

int next_event(lbm_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    c->ev_pool.push_back(e);
  }
  return (int)c->ev_used++;
}

void launch_steps(lbm_ctx* c, int64_t n, int64_t t0) {
  for (int64_t i = 0; i < n; ++i) {
    int parity = (int)((t0 + i) & 1);
    int e0 = -1, e1 = -1, e2 = -1;
    if (c->fused) {
      if (c->profiling) {
        e0 = next_event(c);
        e1 = next_event(c);
      }
      if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], c->stream);
      cudaError_t e = c->fargs.mode == 5   ? c->ops->trailq(c->P, c->f, c->status, c->t_dev, c->fargs, c->stream)
                      : c->fargs.mode == 4 ? c->ops->trail3(c->P, c->f, c->status, c->t_dev, c->fargs, c->stream)
                      : c->fargs.mode == 3 ? c->ops->fused3(c->P, c->f, c->status, c->t_dev, c->fargs, c->stream)
                                           : c->ops->fused(c->P, c->f, c->psi, c->status, c->t_dev, c->fargs, c->stream);
      if (e != cudaSuccess && c->launch_err == cudaSuccess) c->launch_err = e;
      if (e1 >= 0) {
        cudaEventRecord(c->ev_pool[e1], c->stream);
        c->ev_marks[2].push_back({e0, e1});
      }
      continue;
    }
    if (c->profiling) {
      e0 = next_event(c);
      e1 = next_event(c);
      e2 = next_event(c);
    }
    if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], c->stream);
    c->ops->psi(c->P, c->f, c->psi, c->status, parity, c->stream);
    if (e1 >= 0) cudaEventRecord(c->ev_pool[e1], c->stream);
    c->ops->collide(c->P, c->f, c->psi, c->status, c->t_dev, parity, c->stream);
    if (e2 >= 0) {
      cudaEventRecord(c->ev_pool[e2], c->stream);
      c->ev_marks[0].push_back({e0, e1});
      c->ev_marks[1].push_back({e1, e2});
    }
  }
}

void drop_graph(lbm_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  for (auto& g : c->seg_graphs) cudaGraphExecDestroy(g.second);
  c->seg_graphs.clear();
}

void free_fused(lbm_ctx* c) {
  cudaFree(c->fargs.flags);
  cudaFree(c->fargs.done);
  cudaFree(c->fargs.pending);
  cudaFree((void*)c->fargs.range);
  cudaFree((void*)c->fargs.nbr);
  cudaFree(c->fargs.psi_ring);
  cudaFree((void*)c->fargs.tasks);
  cudaFree(c->fargs.ticket);
  c->fargs = lbm::FusedArgs{};
  c->fused = false;
  c->trail_t = -1;
}

// Workers (plane ranges) of the plane-range kernel, or blocks of the tile-column kernel.
int fused_blocks(const lbm_ctx* c) {
  if (c->fargs.mode == 5) return c->fargs.nch;  // k_trailq: chunks of a plane
  return c->fargs.mode >= 3 ? c->fargs.G : c->fargs.ntx * c->fargs.nty * c->fargs.nchunk;
}
// Progress counters of the active fused kernel.
int fused_flags(const lbm_ctx* c) {
  if (c->fargs.mode == 5) return c->fargs.nch * c->P.nz;  // one per (plane, chunk)
  return c->fargs.mode == 3 ? c->fargs.G * c->ops->fused3_flags : fused_blocks(c);
}

// The plane-range fused step (k_fused3, D3Q19): one CTA per SM of ops->fused3_wpc workers,
// G workers in all, worker w owning sites [w nxy / G, (w + 1) nxy / G) of every z plane; the neighbour
// workers of each worker (owners of the 8 in-plane neighbours of its sites) are listed for its
// waits. Returns false when the grid is too small or a worker would have more than kF3MaxNbr
// neighbours.
bool setup_fused3(lbm_ctx* c) {
  if (c->Q != 19 || !c->ops->fused3_max_blocks) return false;
  const int nx = c->P.nx, ny = c->P.ny, nz = c->P.nz;
  const long long nxy = (long long)nx * ny;
  if (nz < 3 || nxy < 64) return false;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int WPC = c->ops->fused3_wpc;
  int G = WPC * (int)std::min<long long>(sms, nxy / 64);  // workers
  int smax = 0;
  bool fits = false;
  for (int tries = 0; tries < 4 && G >= 2; ++tries) {
    smax = (int)((nxy + G - 1) / G);
    const size_t smem = 0;
    const int cap = c->ops->fused3_max_blocks((int)smem);  // co-resident CTAs
    if (cap >= G / WPC) {
      fits = true;
      break;
    }
    if (cap <= 0) return false;
    G = WPC * cap;
  }
  if (!fits) return false;
  std::vector<int> range(G + 1), owner(nxy), nbr((size_t)G * lbm::kF3MaxNbr, -1);
  for (int b = 0; b <= G; ++b) range[b] = (int)((long long)b * nxy / G);
  for (int b = 0; b < G; ++b)
    for (int i = range[b]; i < range[b + 1]; ++i) owner[i] = b;
  for (int b = 0; b < G; ++b) {
    int n = 0;
    for (int i = range[b]; i < range[b + 1]; ++i) {
      const int x = i % nx, y = i / nx;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int o = owner[(size_t)((y + dy + ny) % ny) * nx + (x + dx + nx) % nx];
          if (o == b) continue;
          bool seen = false;
          for (int k = 0; k < n; ++k) seen = seen || nbr[(size_t)b * lbm::kF3MaxNbr + k] == o;
          if (seen) continue;
          if (n == lbm::kF3MaxNbr) return false;
          nbr[(size_t)b * lbm::kF3MaxNbr + n++] = o;
        }
    }
  }
  lbm::FusedArgs a{};
  a.mode = 3;
  a.G = G;
  a.smax = smax;
  a.silent_block = -1;
  int* d_range = nullptr;
  int* d_nbr = nullptr;
  const size_t nflags = (size_t)G * c->ops->fused3_flags;
  bool ok = cudaMalloc(&a.flags, nflags * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&a.done, sizeof(unsigned int)) == cudaSuccess && cudaMalloc(&a.pending, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&d_range, (G + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&d_nbr, nbr.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&a.psi_ring, (size_t)(lbm::kF3Ring + 2) * nxy * c->ops->psi_bytes) == cudaSuccess;
  a.range = d_range;
  a.nbr = d_nbr;
  ok = ok && cudaMemset(a.flags, 0, nflags * sizeof(unsigned long long)) == cudaSuccess &&
       cudaMemset(a.done, 0, sizeof(unsigned int)) == cudaSuccess && cudaMemset(a.pending, 0, sizeof(int)) == cudaSuccess &&
       cudaMemcpy(d_range, range.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
  c->fargs = a;
  if (!ok) {
    cudaGetLastError();
    free_fused(c);
    return false;
  }
  c->fused = true;
  return true;
}

// Chooses the fused tiling: tiles of fused_tx x fused_ty sites across the grid, the slowest
// axis cut into the largest number of chunks (each at least two groups of fused_group planes)
// whose blocks are still all co-resident. Returns false when the grid does not tile or the blocks would not fit.
// The trailing fused step (k_trail3, D3Q19): one CTA per SM (kT3Threads threads), CTA b
// owning sites [b nxy / G, (b + 1) nxy / G) of every z plane, the neighbour CTAs of each CTA
// (owners of the 8 in-plane neighbours of its sites) listed for its waits, and two psi fields.
// Returns false when the grid is too small, a CTA would have more than kF3MaxNbr neighbours or
// the device cannot hold the CTAs at once.
bool setup_trail3(lbm_ctx* c) {
  free_fused(c);
  if (c->Q != 19 || !c->ops->trail3_max_blocks) return false;
  const int nx = c->P.nx, ny = c->P.ny, nz = c->P.nz;
  const long long nxy = (long long)nx * ny;
  if (nz < 3 || nxy < 64) return false;
  const int cap = c->ops->trail3_max_blocks();
  if (cap <= 0) return false;
  const int G = (int)std::min<long long>(cap, nxy / 32);
  if (G < 2) return false;
  std::vector<int> range(G + 1), owner(nxy), nbr((size_t)G * lbm::kF3MaxNbr, -1);
  for (int b = 0; b <= G; ++b) range[b] = (int)((long long)b * nxy / G);
  for (int b = 0; b < G; ++b)
    for (int i = range[b]; i < range[b + 1]; ++i) owner[i] = b;
  for (int b = 0; b < G; ++b) {
    int n = 0;
    for (int i = range[b]; i < range[b + 1]; ++i) {
      const int x = i % nx, y = i / nx;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int o = owner[(size_t)((y + dy + ny) % ny) * nx + (x + dx + nx) % nx];
          if (o == b) continue;
          bool seen = false;
          for (int k = 0; k < n; ++k) seen = seen || nbr[(size_t)b * lbm::kF3MaxNbr + k] == o;
          if (seen) continue;
          if (n == lbm::kF3MaxNbr) return false;
          nbr[(size_t)b * lbm::kF3MaxNbr + n++] = o;
        }
    }
  }
  lbm::FusedArgs a{};
  a.mode = 4;
  a.G = G;
  a.smax = (int)((nxy + G - 1) / G);
  a.silent_block = -1;
  int* d_range = nullptr;
  int* d_nbr = nullptr;
  bool ok = cudaMalloc(&a.flags, (size_t)G * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&a.done, sizeof(unsigned int)) == cudaSuccess && cudaMalloc(&a.pending, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&d_range, (G + 1) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&d_nbr, nbr.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&a.psi_ring, (size_t)2 * c->P.N * c->ops->psi_bytes) == cudaSuccess;
  a.range = d_range;
  a.nbr = d_nbr;
  ok = ok && cudaMemset(a.flags, 0, (size_t)G * sizeof(unsigned long long)) == cudaSuccess &&
       cudaMemset(a.done, 0, sizeof(unsigned int)) == cudaSuccess && cudaMemset(a.pending, 0, sizeof(int)) == cudaSuccess &&
       cudaMemcpy(d_range, range.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
  c->fargs = a;
  if (!ok) {
    cudaGetLastError();
    free_fused(c);
    return false;
  }
  c->fused = true;
  c->trail_t = -1;
  return true;
}

// The task-queue step's schedule (host arithmetic only): chunks of TS consecutive sites of
// the flattened (y, x) index of a plane; nbr[c * kF3MaxNbr ..] the chunks holding the in-plane
// neighbours of chunk c's sites (-1 padded); tasks the ticket order (collision of chunk c of
// plane z: z nch + c; psi of the next step there: -(z nch + c) - 1), every collision in plane
// order with the psi task of (z, c) after the collision of (z + 1 + lag, c) and the psi tasks
// the march does not place (planes nz - 1 and 0 among them) at the end, plane 0 last. Checks
// that every collision a psi task needs (planes z - 1 .. z + 1 of the chunk and its neighbour
// chunks) has a smaller ticket. Returns the chunks per plane, or -1 for a grid it does not serve.
int queue_schedule(int nx, int ny, int nz, int TS, int lag, std::vector<int>& nbr, std::vector<int>& tasks) {
  const long long nxy = (long long)nx * ny;
  if (nx < 1 || ny < 1 || nz < 3 || TS < 1 || lag < 1) return -1;
  const int nch = (int)((nxy + TS - 1) / TS);
  if ((long long)nch * nz * 2 >= (1LL << 30)) return -1;
  const int K = lbm::kF3MaxNbr;
  nbr.assign((size_t)nch * K, -1);
  for (int ch = 0; ch < nch; ++ch) {
    int n = 0;
    const long long hi = std::min<long long>((long long)(ch + 1) * TS, nxy);
    for (long long i = (long long)ch * TS; i < hi; ++i) {
      const int x = (int)(i % nx), y = (int)(i / nx);
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int o = (int)((((long long)((y + dy + ny) % ny)) * nx + (x + dx + nx) % nx) / TS);
          if (o == ch) continue;
          bool seen = false;
          for (int k = 0; k < n; ++k) seen = seen || nbr[(size_t)ch * K + k] == o;
          if (seen) continue;
          if (n == K) return -1;
          nbr[(size_t)ch * K + n++] = o;
        }
    }
  }
  const long long ncol = (long long)nz * nch;
  tasks.clear();
  tasks.reserve((size_t)(2 * ncol));
  std::vector<char> placed((size_t)ncol, 0);
  for (long long i = 0; i < ncol; ++i) {
    tasks.push_back((int)i);
    const long long zp = i / nch - 1 - lag, cp = i % nch;
    if (zp >= 1 && zp <= nz - 2) {
      tasks.push_back((int)(-(zp * nch + cp) - 1));
      placed[(size_t)(zp * nch + cp)] = 1;
    }
  }
  for (int z = 1; z < nz; ++z)
    for (int ch = 0; ch < nch; ++ch)
      if (!placed[(size_t)z * nch + ch]) tasks.push_back(-(z * nch + ch) - 1);
  for (int ch = 0; ch < nch; ++ch) tasks.push_back(-ch - 1);
  std::vector<long long> pos((size_t)ncol, -1);
  for (size_t p = 0; p < tasks.size(); ++p)
    if (tasks[p] >= 0) pos[(size_t)tasks[p]] = (long long)p;
  for (size_t p = 0; p < tasks.size(); ++p) {
    if (tasks[p] >= 0) continue;
    const int q = -tasks[p] - 1, z = q / nch, ch = q % nch;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = (z + dz + nz) % nz;
      for (int j = -1; j < K && (j < 0 || nbr[(size_t)ch * K + j] >= 0); ++j) {
        const int cc = j < 0 ? ch : nbr[(size_t)ch * K + j];
        const long long pc = pos[(size_t)zz * nch + cc];
        if (pc < 0 || pc >= (long long)p) return -1;
      }
    }
  }
  return nch;
}

// The task-queue one-pass step (k_trailq, D3Q19): each plane cut into nch chunks of
// ops->trailq_chunk consecutive sites of the flattened (y, x) index; per chunk the chunks
// holding the in-plane neighbours of its sites; the ticket order of the step's tasks (every
// collision in plane order, the psi task of (z, c) after the collision of (z + 1 + lag, c), the
// psi tasks of planes nz - 1 and 0 last), checked here to place every task a psi task waits for
// at a smaller ticket; one progress flag per (plane, chunk); two psi fields. As many CTAs as
// the device holds at once (fewer would also be correct: see the kernel's header).
bool setup_trailq(lbm_ctx* c) {
  free_fused(c);
  if (c->Q != 19 || !c->ops->trailq_max_blocks) return false;
  const int nx = c->P.nx, ny = c->P.ny, nz = c->P.nz;
  const long long nxy = (long long)nx * ny;
  if (nz < 3 || nxy < 1) return false;
  const int cap = c->ops->trailq_max_blocks();
  if (cap <= 0) return false;
  const int TS = (int)std::min<long long>(c->ops->trailq_chunk, nxy);
  std::vector<int> nbr, tasks;
  const int nch = queue_schedule(nx, ny, nz, TS, c->ops->trailq_lag, nbr, tasks);
  if (nch < 0) return false;
  const long long ncol = (long long)nz * nch;
  lbm::FusedArgs a{};
  a.mode = 5;
  a.G = (int)std::min<long long>(cap, (long long)tasks.size());
  a.smax = TS;
  a.nch = nch;
  a.ntask = (int)tasks.size();
  a.silent_block = -1;
  int* d_nbr = nullptr;
  int* d_tasks = nullptr;
  bool ok = cudaMalloc(&a.flags, (size_t)ncol * sizeof(unsigned long long)) == cudaSuccess &&
            cudaMalloc(&a.done, sizeof(unsigned int)) == cudaSuccess && cudaMalloc(&a.pending, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&a.ticket, sizeof(unsigned int)) == cudaSuccess &&
            cudaMalloc(&d_nbr, nbr.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&d_tasks, tasks.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&a.psi_ring, (size_t)2 * c->P.N * c->ops->psi_bytes) == cudaSuccess;
  a.nbr = d_nbr;
  a.tasks = d_tasks;
  ok = ok && cudaMemset(a.flags, 0, (size_t)ncol * sizeof(unsigned long long)) == cudaSuccess &&
       cudaMemset(a.done, 0, sizeof(unsigned int)) == cudaSuccess && cudaMemset(a.pending, 0, sizeof(int)) == cudaSuccess &&
       cudaMemset(a.ticket, 0, sizeof(unsigned int)) == cudaSuccess &&
       cudaMemcpy(d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(d_tasks, tasks.data(), tasks.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess;
  c->fargs = a;
  if (!ok) {
    cudaGetLastError();
    free_fused(c);
    return false;
  }
  c->fused = true;
  c->trail_t = -1;
  return true;
}

bool setup_fused(lbm_ctx* c) {
  free_fused(c);
  if (setup_fused3(c)) return true;
  const int TX = c->ops->fused_tx, TY = c->ops->fused_ty;
  const bool d3 = c->Q == 19;
  const int nx = c->P.nx, ny = c->P.ny, nz = c->P.nz;
  const int nm = d3 ? nz : ny;
  if (nx % TX != 0 || (d3 && ny % TY != 0)) return false;
  const int ntx = nx / TX, nty = d3 ? ny / TY : 1;
  const int cap = c->ops->fused_max_blocks();
  const long long tiles = (long long)ntx * nty;
  const int NP = c->ops->fused_group;
  int best = 0;
  for (int nch = 1; nch <= nm; ++nch)
    if (nm % (nch * NP) == 0 && nm / (nch * NP) >= 2 && tiles * nch <= cap) best = nch;
  if (best == 0) return false;
  const size_t nb = (size_t)tiles * best;
  lbm::FusedArgs a{};
  a.ntx = ntx;
  a.nty = nty;
  a.nchunk = best;
  a.L = nm / best;
  a.silent_block = -1;
  if (cudaMalloc(&a.flags, nb * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMalloc(&a.done, sizeof(unsigned int)) != cudaSuccess || cudaMalloc(&a.pending, sizeof(int)) != cudaSuccess ||
      cudaMemset(a.flags, 0, nb * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMemset(a.done, 0, sizeof(unsigned int)) != cudaSuccess || cudaMemset(a.pending, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    c->fargs = a;
    free_fused(c);
    return false;
  }
  c->fargs = a;
  c->fused = true;
  return true;
}

// The path LBM_PATH_AUTO takes: the two-kernel step, the faster one measured on GB300 for
// both lattices (D3Q19 at 256^3, three FP32-shifted components: 2.11 ms against 3.48 ms for
// the plane-range fused form, whose collision runs at 14 warps per SM with register spills and
// per-plane synchronisation; D2Q9 at 512^2, three components, MRT: 22.8 us against 33.5 us,
// and at 256^2, two components, BGK: 8.2 us against 22.5 us for the tile-column form).
bool setup_auto(lbm_ctx* c) {
  free_fused(c);
  return false;
}

// Progress counters must not exceed t * L when the step counter is reset or rewound.
cudaError_t reset_fused_flags(lbm_ctx* c) {
  if (!c->fused) return cudaSuccess;
  return cudaMemsetAsync(c->fargs.flags, 0, (size_t)fused_flags(c) * sizeof(unsigned long long), c->stream);
}

// Captures kGraphSteps steps starting at an even step; on any capture failure the context
// falls back to direct launches for good.
bool build_graph(lbm_ctx* c) {
  if (c->graph) return true;
  if (c->graph_failed || c->stream == nullptr) return false;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->graph_failed = true;
    return false;
  }
  launch_steps(c, kGraphSteps, 0);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess || !g) {
    cudaGetLastError();
    c->graph_failed = true;
    return false;
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->graph = nullptr;
    c->graph_failed = true;
    return false;
  }
  return true;
}

// The captured graph of n steps starting at a step of the given parity (lbm_record's
// segments), or nullptr when capture is not possible (the caller launches directly).
cudaGraphExec_t segment_graph(lbm_ctx* c, int64_t n, int parity) {
  for (auto& g : c->seg_graphs)
    if (g.first.first == n && g.first.second == parity) return g.second;
  if (c->graph_failed || c->stream == nullptr || c->seg_graphs.size() >= 8) return nullptr;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  launch_steps(c, n, parity);
  cudaGraphExec_t x = nullptr;
  if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess || !g || cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return nullptr;
  }
  cudaGraphDestroy(g);
  c->seg_graphs.push_back({{n, parity}, x});
  return x;
}

}  // namespace

namespace lbm {

// Validates one lattice description and fills its kernel parameters (Section 3.2 component
// parameters, mixing-rule products, MRT rates) and dispatch table. Touches no device state.
lbm_status make_params(const lbm_grid* grid, int nc, const lbm_component* comps, const lbm_eos* eos, double tau,
                       Params* out, const Ops** ops_out, std::string* why) {
  auto bad = [&](const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    *why = buf;
    return LBM_ERR_ARG;
  };
  if (!grid || !comps || !eos) return bad("grid, comps and eos must be non-NULL");
  if (grid->lattice != LBM_D2Q9 && grid->lattice != LBM_D3Q19)
    return bad("lattice must be 9 (D2Q9) or 19 (D3Q19)");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return bad("grid sizes must be >= 1");
  if (grid->lattice == LBM_D2Q9 && grid->nz != 1) return bad("D2Q9 needs nz == 1");
  const int64_t N = (int64_t)grid->nx * grid->ny * grid->nz;
  if (N * grid->lattice >= ((int64_t)1 << 32))
    return bad("grid too large: Q * nx * ny * nz must stay below 2^32 (226 M D3Q19 sites)");
  if (nc < 1 || nc > 4) return bad("nc must be 1..4");
  if (!(tau > 0.5) || !std::isfinite(tau)) return bad("tau must be > 1/2");
  if (eos->precision != LBM_FP64 && eos->precision != LBM_FP32_SHIFTED)
    return bad("precision must be LBM_FP64 or LBM_FP32_SHIFTED");
  if (eos->collision != LBM_BGK && eos->collision != LBM_MRT)
    return bad("collision must be LBM_BGK or LBM_MRT");
  if (eos->collision == LBM_MRT && !eos->mrt_rates) return bad("MRT needs mrt_rates");
  if (!(eos->T > 0) || !std::isfinite(eos->T)) return bad("T must be > 0");
  if (!(eos->G != 0) || !std::isfinite(eos->G)) return bad("G must be nonzero");
  if (!std::isfinite(eos->beta)) return bad("beta must be finite");
  if (eos->split != LBM_SPLIT_VOLATILITY && eos->split != LBM_SPLIT_GONG) return bad("split must be 0 or 1");
  const double R = eos->R == 0 ? 1.0 : eos->R;
  if (!(R > 0) || !std::isfinite(R)) return bad("R must be > 0");
  for (int i = 0; i < nc; ++i) {
    const lbm_component& k = comps[i];
    if (!(k.Tc > 0) || !(k.pc > 0) || !(k.M > 0) || !std::isfinite(k.omega) || !std::isfinite(k.Tc) ||
        !std::isfinite(k.pc) || !std::isfinite(k.M))
      return bad("component %d: Tc, pc, M must be finite and > 0", i);
    if (eos->gamma && (!(eos->gamma[i] > 0) || !std::isfinite(eos->gamma[i])))
      return bad("gamma[%d] must be finite and > 0", i);
    if (eos->rho_ref && !std::isfinite(eos->rho_ref[i]))
      return bad("rho_ref[%d] must be finite", i);
    if (eos->kij)
      for (int j = 0; j < nc; ++j)
        if (!std::isfinite(eos->kij[i * nc + j]) || eos->kij[i * nc + j] != eos->kij[j * nc + i])
          return bad("kij must be finite and symmetric");
  }
  const int Q = grid->lattice;
  if (eos->collision == LBM_MRT)
    for (int k = 0; k < Q; ++k)
      if (!std::isfinite(eos->mrt_rates[k]) || !(eos->mrt_rates[k] > 0) || !(eos->mrt_rates[k] < 2))
        return bad("mrt_rates[%d] must lie in (0, 2)", k);
  const Ops* ops = ops_get(Q, eos->precision == LBM_FP32_SHIFTED, eos->collision == LBM_MRT, nc);
  if (!ops) return bad("no kernels for this configuration");

  Params& P = *out;
  P = Params{};
  P.nx = grid->nx;
  P.ny = grid->ny;
  P.nz = grid->nz;
  P.N = N;
  P.N32 = (uint32_t)N;
  P.nc = nc;
  P.omega = 1.0 / tau;
  for (int i = 0; i < nk_q(Q); ++i) {
    int k = rows_q(Q, i);
    P.lam[i] = eos->collision == LBM_MRT ? (eos->mrt_rates[k] - P.omega) / norm_q(Q, k) : 0.0;
  }
  // Section 3.2: a_i = Omega_a R^2 Tc^2 / pc, b_i = Omega_b R Tc / pc, alpha_i(T), m_i
  double aa[4];
  for (int i = 0; i < nc; ++i) {
    const lbm_component& k = comps[i];
    double sq = 1.0 + m_factor(k.omega) * (1.0 - std::sqrt(eos->T / k.Tc));
    aa[i] = kOmegaA * R * R * k.Tc * k.Tc / k.pc * sq * sq;
    P.b[i] = kOmegaB * R * k.Tc / k.pc;
    P.invM[i] = 1.0 / k.M;
    P.gamma[i] = eos->gamma ? eos->gamma[i] : 1.0;
    P.rho_ref[i] = (eos->precision == LBM_FP32_SHIFTED && eos->rho_ref) ? eos->rho_ref[i] : 0.0;
  }
  P.kij_zero = 1;
  for (int i = 0; i < nc; ++i) {
    P.sa[i] = std::sqrt(aa[i]);
    P.invMf[i] = (float)(1.0 / comps[i].M);
    for (int j = 0; j < nc; ++j) {
      const double k = eos->kij ? eos->kij[i * nc + j] : 0.0;
      if (k != 0.0) P.kij_zero = 0;
      P.Qa[i * 4 + j] = std::sqrt(aa[i] * aa[j]) * (1.0 - k);
    }
  }
  P.RT = R * eos->T;
  P.cpsi = 2.0 / (eos->G * (1.0 / 3.0));
  P.beta = eos->beta;
  P.split = eos->split;
  P.G = eos->G;
  finalize_params(P);
  *ops_out = ops;
  return LBM_OK;
}

}  // namespace lbm


extern "C" {

lbm_status lbm_create(const lbm_grid* grid, int nc, const lbm_component* comps, const lbm_eos* eos,
                      double tau, lbm_ctx** out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  lbm::Params P{};
  const lbm::Ops* ops = nullptr;
  std::string why;
  lbm_status st = lbm::make_params(grid, nc, comps, eos, tau, &P, &ops, &why);
  if (st != LBM_OK) return fail(nullptr, st, "%s", why.c_str());
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(nullptr, LBM_ERR_OOM, "host allocation failed");
  c->grid = *grid;
  c->nc = nc;
  c->Q = grid->lattice;
  c->precision = eos->precision;
  c->collision = eos->collision;
  c->ops = ops;
  c->P = P;
  c->ref_given = eos->rho_ref != nullptr;
  const int Q = c->Q;
  const int64_t N = P.N;

  cudaError_t e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&c->f, (size_t)nc * Q * N * ops->store_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->psi, (size_t)N * ops->psi_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&c->t_dev, sizeof(long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->partial, (size_t)((N + 255) / 256) * nc * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->mass_dev, 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->t_dev, 0, sizeof(long long));
  if (e != cudaSuccess) {
    lbm_status st = cuda_fail(nullptr, e, "lbm_create allocation");
    lbm_destroy(c);
    return st;
  }
  c->stream = c->own;
  setup_auto(c);
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  free_fused(c);
  cudaFree(c->ckpt_base);
  cudaFree(c->f);
  cudaFree(c->psi);
  cudaFree(c->status);
  cudaFree(c->t_dev);
  cudaFree(c->partial);
  cudaFree(c->mass_dev);
  cudaFree(c->scratch);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
}

lbm_status lbm_profile(lbm_ctx* c, int on) {
  if (!c) return LBM_ERR_ARG;
  CK(c, cudaStreamSynchronize(c->stream));
  c->profiling = on != 0;
  c->ev_used = 0;
  c->ev_marks[0].clear();
  c->ev_marks[1].clear();
  c->ev_marks[2].clear();
  return LBM_OK;
}

lbm_status lbm_profile_read(lbm_ctx* c, int kernel, double* total_ms, int64_t* launches) {
  if (!c || kernel < 0 || kernel > 2) return c ? fail(c, LBM_ERR_ARG, "kernel must be 0, 1 or 2") : LBM_ERR_ARG;
  CK(c, cudaStreamSynchronize(c->stream));
  double sum = 0;
  for (auto& m : c->ev_marks[kernel]) {
    float ms = 0;
    CK(c, cudaEventElapsedTime(&ms, c->ev_pool[m.first], c->ev_pool[m.second]));
    sum += ms;
  }
  if (total_ms) *total_ms = sum;
  if (launches) *launches = (int64_t)c->ev_marks[kernel].size();
  return LBM_OK;
}

lbm_status lbm_set_stream(lbm_ctx* c, void* stream) {
  if (!c) return LBM_ERR_ARG;
  CK(c, cudaStreamSynchronize(c->stream));
  drop_graph(c);
  c->graph_failed = false;
  c->stream = stream ? (cudaStream_t)stream : c->own;
  return LBM_OK;
}

lbm_status lbm_init(lbm_ctx* c, const double* rho, const double* u) {
  if (!c) return LBM_ERR_ARG;
  if (!rho) return fail(c, LBM_ERR_ARG, "rho is NULL");
  const int64_t N = c->P.N;
  lbm_status st = ensure_scratch(c);
  if (st != LBM_OK) return st;
  double* d_rho = c->scratch;
  double* d_u = c->scratch + (size_t)c->nc * N;
  unsigned long long* d_chk = (unsigned long long*)(c->scratch + (size_t)(c->nc + 5) * N);
  // page-locked inputs are read in place by the kernels (this call synchronises before it
  // returns); others are copied to device memory first
  if (const double* m = mapped_range(rho, (size_t)c->nc * N))
    d_rho = const_cast<double*>(m);
  else
    CK(c, copy_in(d_rho, rho, (size_t)c->nc * N * sizeof(double), c->stream));
  if (u) {
    if (const double* m = mapped_range(u, (size_t)3 * N))
      d_u = const_cast<double*>(m);
    else
      CK(c, copy_in(d_u, u, (size_t)3 * N * sizeof(double), c->stream));
  }
  // densities finite and > 0, u finite, and the component minima (the default FP32 shift)
  unsigned long long chk[6];
  CK(c, cudaMemsetAsync(d_chk, 0xff, 5 * sizeof(unsigned long long), c->stream));
  CK(c, cudaMemsetAsync(d_chk + 5, 0, sizeof(unsigned long long), c->stream));
  const long long work = (long long)c->nc * N;
  const unsigned nb = (unsigned)std::min<long long>((work + 255) / 256, 4096);
  k_check_init<<<nb, 256, 0, c->stream>>>(d_rho, u ? d_u : nullptr, (long long)N, c->nc, d_chk);
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(chk, d_chk, sizeof chk, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (chk[4] != ~0ull)
    return fail(c, LBM_ERR_ARG, "rho[%d][%lld] must be finite and > 0", (int)(chk[4] / (unsigned long long)N),
                (long long)(chk[4] % (unsigned long long)N));
  if (chk[5]) return fail(c, LBM_ERR_ARG, "u must be finite");
  if (c->precision == LBM_FP32_SHIFTED && !c->ref_given) {
    for (int s = 0; s < c->nc; ++s) {
      double lo;
      std::memcpy(&lo, &chk[s], sizeof lo);
      c->P.rho_ref[s] = lo;
    }
    lbm::finalize_params(c->P);
    drop_graph(c);  // the graph holds the parameters by value
  }
  c->ops->init(c->P, c->f, d_rho, u ? d_u : nullptr, c->stream);
  CK(c, cudaGetLastError());
  CK(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CK(c, cudaMemsetAsync(c->t_dev, 0, sizeof(long long), c->stream));
  CK(c, reset_fused_flags(c));
  CK(c, cudaStreamSynchronize(c->stream));
  c->t = 0;
  c->trail_t = -1;
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t n) {
  if (!c) return LBM_ERR_ARG;
  if (n < 0) return fail(c, LBM_ERR_ARG, "n must be >= 0");
  int64_t t = c->t, left = n;
  const bool trailing = c->fused && c->fargs.mode >= 4;
  if (trailing && n > 0 && c->trail_t != t) {
    // psi of the first step, which the trailing step reads from psi_ring[t & 1]
    const int e0 = c->profiling ? next_event(c) : -1, e1 = c->profiling ? next_event(c) : -1;
    if (e0 >= 0) cudaEventRecord(c->ev_pool[e0], c->stream);
    c->ops->psi(c->P, c->f, (char*)c->fargs.psi_ring + (size_t)(t & 1) * c->P.N * c->ops->psi_bytes, c->status,
                (int)(t & 1), c->stream);
    if (e1 >= 0) {
      cudaEventRecord(c->ev_pool[e1], c->stream);
      c->ev_marks[0].push_back({e0, e1});
    }
  }
  if (!trailing) c->trail_t = -1;
  if ((t & 1) && left > 0) {  // reach an even step before replaying graphs
    launch_steps(c, 1, t);
    ++t;
    --left;
  }
  while (!c->profiling && left >= kGraphSteps && build_graph(c)) {
    CK(c, cudaGraphLaunch(c->graph, c->stream));
    t += kGraphSteps;
    left -= kGraphSteps;
  }
  launch_steps(c, left, t);
  c->trail_t = -1;
  if (c->launch_err != cudaSuccess) {
    cudaError_t e = c->launch_err;
    c->launch_err = cudaSuccess;
    cudaStreamSynchronize(c->stream);
    return cuda_fail(c, e, "fused step launch");
  }
  CK(c, cudaGetLastError());
  lbm_status st = sync_status(c);
  if (st == LBM_OK && trailing) c->trail_t = c->t;
  return st;
}

lbm_status lbm_set_path(lbm_ctx* c, int path) {
  if (!c) return LBM_ERR_ARG;
  if (path != LBM_PATH_AUTO && path != LBM_PATH_TWO_KERNEL && path != LBM_PATH_FUSED && path != LBM_PATH_TRAILING &&
      path != LBM_PATH_QUEUE)
    return fail(c, LBM_ERR_ARG, "unknown path %d", path);
  CK(c, cudaStreamSynchronize(c->stream));
  drop_graph(c);
  c->graph_failed = false;
  c->path_request = path;
  if (path == LBM_PATH_TWO_KERNEL) {
    free_fused(c);
    return LBM_OK;
  }
  if (path == LBM_PATH_AUTO) {
    setup_auto(c);
    return LBM_OK;
  }
  if (path == LBM_PATH_TRAILING) {
    if (!setup_trail3(c))
      return fail(c, LBM_ERR_ARG, "the trailing step needs D3Q19, nz >= 3 and co-resident CTAs for this grid");
    return LBM_OK;
  }
  if (path == LBM_PATH_QUEUE) {
    if (!setup_trailq(c))
      return fail(c, LBM_ERR_ARG, "the task-queue step needs D3Q19 and nz >= 3");
    return LBM_OK;
  }
  if (!setup_fused(c))
    return fail(c, LBM_ERR_ARG, "the fused step does not fit this grid (tiles %dx%d, co-residency)",
                c->ops->fused_tx, c->ops->fused_ty);
  return LBM_OK;
}

lbm_status lbm_test_silence_block(lbm_ctx* c, int block) {
  if (!c) return LBM_ERR_ARG;
  if (!c->fused) return fail(c, LBM_ERR_ARG, "the fused path is not active");
  const int nb = fused_blocks(c);
  if (block < -1 || block >= nb) return fail(c, LBM_ERR_ARG, "block must be -1 or in [0, %d)", nb);
  CK(c, cudaStreamSynchronize(c->stream));
  drop_graph(c);
  c->fargs.silent_block = block;
  return LBM_OK;
}

int lbm_get_path(const lbm_ctx* c) {
  if (!c) return -1;
  if (!c->fused) return LBM_PATH_TWO_KERNEL;
  if (c->fargs.mode == 5) return LBM_PATH_QUEUE;
  return c->fargs.mode == 4 ? LBM_PATH_TRAILING : LBM_PATH_FUSED;
}

int lbm_get_fused_kind(const lbm_ctx* c) {
  if (!c || !c->fused || c->fargs.mode >= 4) return 0;
  return c->fargs.mode == 3 ? LBM_FUSED_PLANES : LBM_FUSED_TILES;
}

int64_t lbm_time(const lbm_ctx* c) { return c ? c->t : -1; }

lbm_status lbm_fields(lbm_ctx* c, double* rho, double* u, double* p, double* psi) {
  if (!c) return LBM_ERR_ARG;
  lbm_status st = ensure_scratch(c);
  if (st != LBM_OK) return st;
  const int64_t N = c->P.N;
  double* d_rho = c->scratch;
  double* d_u = d_rho + (size_t)c->nc * N;
  double* d_p = d_u + (size_t)3 * N;
  double* d_psi = d_p + N;
  const int parity = (int)(c->t & 1);
  // page-locked outputs are written in place by the kernel (this call synchronises before it
  // returns); others are staged in device memory and copied back
  double* m_rho = mapped_range(rho, (size_t)c->nc * N);
  double* m_u = mapped_range(u, (size_t)3 * N);
  double* m_p = mapped_range(p, (size_t)N);
  double* m_psi = mapped_range(psi, (size_t)N);
  if (u || psi) c->ops->psi(c->P, c->f, c->psi, c->status, parity, c->stream);  // the state's psi
  c->ops->fields(c->P, c->f, c->psi, rho ? (m_rho ? m_rho : d_rho) : nullptr, u ? (m_u ? m_u : d_u) : nullptr,
                 p ? (m_p ? m_p : d_p) : nullptr, psi ? (m_psi ? m_psi : d_psi) : nullptr, parity, c->stream);
  CK(c, cudaGetLastError());
  if (rho && !m_rho) CK(c, copy_out(rho, d_rho, (size_t)c->nc * N * sizeof(double), c->stream));
  if (u && !m_u) CK(c, copy_out(u, d_u, (size_t)3 * N * sizeof(double), c->stream));
  if (p && !m_p) CK(c, copy_out(p, d_p, (size_t)N * sizeof(double), c->stream));
  if (psi && !m_psi) CK(c, copy_out(psi, d_psi, (size_t)N * sizeof(double), c->stream));
  int64_t t = c->t;
  st = sync_status(c);
  c->t = t;
  return st;
}

lbm_status lbm_diagnostics(lbm_ctx* c, const lbm_diag_params* dp, lbm_diag_result* out) {
  if (!c) return LBM_ERR_ARG;
  if (!dp || !out) return fail(c, LBM_ERR_ARG, "params and out must be non-NULL");
  if (dp->erode < 0 || !std::isfinite(dp->threshold)) return fail(c, LBM_ERR_ARG, "erode must be >= 0 and threshold finite");
  lbm_status st = ensure_scratch(c);
  if (st != LBM_OK) return st;
  const int64_t N = c->P.N;
  double* d_rho = c->scratch;
  double* d_p = d_rho + (size_t)(c->nc + 3) * N;
  c->ops->fields(c->P, c->f, c->psi, d_rho, nullptr, d_p, nullptr, (int)(c->t & 1), c->stream);
  CK(c, cudaGetLastError());
  void* work = nullptr;
  CK(c, cudaMallocAsync(&work, (size_t)12 * N + 256, c->stream));
  std::string why;
  st = lbm::diagnostics(c->P, c->nc, c->Q == 19 ? 3 : 2, dp, d_rho, d_p, work, c->stream, out, &why);
  cudaFreeAsync(work, c->stream);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (st != LBM_OK) return fail(c, st, "diagnostics: %s", why.c_str());
  CK(c, e);
  return LBM_OK;
}

lbm_status lbm_mass(lbm_ctx* c, double* mass) {
  if (!c || !mass) return c ? fail(c, LBM_ERR_ARG, "mass is NULL") : LBM_ERR_ARG;
  c->ops->mass(c->P, c->f, c->partial, c->mass_dev, c->stream);
  CK(c, cudaGetLastError());
  CK(c, cudaMemcpyAsync(mass, c->mass_dev, (size_t)c->nc * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_get_f(lbm_ctx* c, double* f) {
  if (!c || !f) return c ? fail(c, LBM_ERR_ARG, "f is NULL") : LBM_ERR_ARG;
  const int64_t N = c->P.N;
  double* d = nullptr;
  const size_t bytes = (size_t)c->nc * c->Q * N * sizeof(double);
  CK(c, cudaMallocAsync(&d, bytes, c->stream));
  c->ops->get_f(c->P, c->f, d, (int)(c->t & 1), c->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(d, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_f");
  return LBM_OK;
}

lbm_status lbm_set_f(lbm_ctx* c, const double* f) {
  if (!c || !f) return c ? fail(c, LBM_ERR_ARG, "f is NULL") : LBM_ERR_ARG;
  const int64_t N = c->P.N;
  const size_t n = (size_t)c->nc * c->Q * N;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(f[i])) return fail(c, LBM_ERR_ARG, "f must be finite");
  double* d = nullptr;
  CK(c, cudaMallocAsync(&d, n * sizeof(double), c->stream));
  cudaError_t e = cudaMemcpyAsync(d, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    c->ops->set_f(c->P, c->f, d, c->stream);
    e = cudaGetLastError();
  }
  cudaFreeAsync(d, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->t_dev, 0, sizeof(long long), c->stream);
  if (e == cudaSuccess) e = reset_fused_flags(c);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->trail_t = -1;
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_f");
  c->t = 0;
  return LBM_OK;
}

size_t lbm_state_bytes(const lbm_ctx* c) {
  return c ? (size_t)c->nc * c->Q * (size_t)c->P.N * c->ops->store_bytes : 0;
}

lbm_status lbm_save(lbm_ctx* c, void* buf, size_t bytes, int64_t* t) {
  if (!c || !buf) return c ? fail(c, LBM_ERR_ARG, "buf is NULL") : LBM_ERR_ARG;
  if (bytes != lbm_state_bytes(c)) return fail(c, LBM_ERR_ARG, "bytes must equal lbm_state_bytes");
  CK(c, cudaMemcpyAsync(buf, c->f, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (t) *t = c->t;
  return LBM_OK;
}

lbm_status lbm_restore(lbm_ctx* c, const void* buf, size_t bytes, int64_t t) {
  if (!c || !buf) return c ? fail(c, LBM_ERR_ARG, "buf is NULL") : LBM_ERR_ARG;
  if (bytes != lbm_state_bytes(c)) return fail(c, LBM_ERR_ARG, "bytes must equal lbm_state_bytes");
  if (t < 0) return fail(c, LBM_ERR_ARG, "t must be >= 0");
  CK(c, cudaMemcpyAsync(c->f, buf, bytes, cudaMemcpyHostToDevice, c->stream));
  long long tt = t;
  CK(c, cudaMemcpyAsync(c->t_dev, &tt, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
  c->trail_t = -1;
  CK(c, cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
  CK(c, reset_fused_flags(c));
  CK(c, cudaStreamSynchronize(c->stream));
  c->t = t;
  return LBM_OK;
}

lbm_status lbm_record(lbm_ctx* c, int64_t n, int checkpoint_every) {
  if (!c) return LBM_ERR_ARG;
  if (c->P.split != LBM_SPLIT_VOLATILITY)
    return fail(c, LBM_ERR_ARG, "the adjoint covers the volatility split (Eq. distributionforce) only");
  if (n < 1 || checkpoint_every < 1) return fail(c, LBM_ERR_ARG, "n and checkpoint_every must be >= 1");
  c->ckpt.clear();
  c->rec_t0 = -1;
  const size_t bytes = lbm_state_bytes(c);
  const int64_t t0 = c->t;
  const int64_t nseg = (n + checkpoint_every - 1) / checkpoint_every;
  // one allocation for every checkpoint, kept for later recordings of the same size or less
  const size_t need = (size_t)nseg * bytes;
  if (c->ckpt_bytes < need) {
    cudaFree(c->ckpt_base);
    c->ckpt_base = nullptr;
    c->ckpt_bytes = 0;
    CK(c, cudaMalloc(&c->ckpt_base, need));
    c->ckpt_bytes = need;
  }
  // the segments run back to back on the stream, each a captured graph of its steps (by step
  // count and parity of its first step) after a copy of its starting state; the stream is
  // synchronised once at the end. The trailing step keeps psi between steps and is driven
  // through lbm_step instead.
  const bool trailing = c->fused && c->fargs.mode >= 4;
  for (int64_t done = 0, i = 0; done < n; ++i) {
    void* p = (char*)c->ckpt_base + (size_t)i * bytes;
    c->ckpt.push_back(p);
    CK(c, cudaMemcpyAsync(p, c->f, bytes, cudaMemcpyDeviceToDevice, c->stream));
    const int64_t k = std::min<int64_t>(checkpoint_every, n - done);
    if (trailing) {
      lbm_status st = lbm_step(c, k);
      if (st != LBM_OK) return st;
    } else {
      cudaGraphExec_t g = c->profiling ? nullptr : segment_graph(c, k, (int)((t0 + done) & 1));
      if (g)
        CK(c, cudaGraphLaunch(g, c->stream));
      else
        launch_steps(c, k, t0 + done);
    }
    done += k;
  }
  if (!trailing) {
    CK(c, cudaGetLastError());
    lbm_status st = sync_status(c);
    if (st != LBM_OK) return st;
  }
  c->trail_t = -1;
  c->ck_every = checkpoint_every;
  c->rec_t0 = t0;
  c->rec_n = n;
  return LBM_OK;
}

namespace {

// beta(c, r) = C(c + r, c): the most steps that c state snapshots, the one holding the start
// included, reverse with every step advanced at most r times (binomial checkpointing;
// saturates at 2^40). beta(c, r) = beta(c, r - 1) + beta(c - 1, r), beta(1, r) = r + 1.
int64_t beta_cr(int c, int r) {
  double b = 1.0;
  for (int i = 1; i <= c; ++i) b = b * (double)(r + i) / (double)i;
  return b > 1099511627776.0 ? (int64_t)1099511627776 : (int64_t)(b + 0.5);
}
// Fewest forward steps that reverse l steps with c snapshots (the start's included):
// t(l, c) = r l - beta(c + 1, r - 1) for beta(c, r - 1) < l <= beta(c, r) (Griewank's binomial
// checkpointing); t(l, 1) = l (l - 1) / 2.
int64_t revolve_min(int64_t l, int c) {
  if (l <= 1) return 0;
  if (c <= 1) return l * (l - 1) / 2;
  int r = 0;
  while (beta_cr(c, r) < l) ++r;
  return (int64_t)r * l - beta_cr(c + 1, r - 1);
}
// First advance of an optimal reversal of n >= 2 steps with s >= 1 free slots besides the one
// holding the start (c = s + 1 snapshots): the m whose split attains the least total,
// m + t(n - m, c - 1) + t(m, c) = t(n, c), searched over the binomial interval
// [n - beta(c - 1, r), beta(c, r - 1)] (the right part reversible with c - 1 snapshots, the left
// part with c snapshots and one repetition fewer), r the least with beta(c, r) >= n.
int64_t binomial_split(int64_t n, int s) {
  const int c = s + 1;
  int r = 0;
  while (beta_cr(c, r) < n) ++r;
  int64_t lo = std::max<int64_t>(1, n - beta_cr(c - 1, r));
  int64_t hi = std::min<int64_t>(n - 1, r > 0 ? beta_cr(c, r - 1) : 1);
  if (hi < lo) hi = lo;
  const int64_t best = revolve_min(n, c);
  int64_t arg = lo, val = -1;
  for (int64_t m = lo; m <= hi; ++m) {
    const int64_t v = m + revolve_min(n - m, c - 1) + revolve_min(m, c);
    if (v == best) return m;
    if (val < 0 || v < val) {
      val = v;
      arg = m;
    }
  }
  return arg;
}

}  // namespace

int64_t revolve_count(int64_t n, int s) {
  if (n <= 1) return 0;
  if (s == 0) return n * (n - 1) / 2;
  const int64_t m = binomial_split(n, s);
  return m + revolve_count(n - m, s - 1) + revolve_count(m, s);
}

static_assert(lbm::kF3MaxNbr == LBM_QUEUE_MAX_NBR, "neighbour-chunk list length of lbm_queue_schedule");

int lbm_queue_schedule(int nx, int ny, int nz, int chunk, int lag, int* nbr, int* tasks) {
  if (nx < 1 || ny < 1) return -1;
  if (chunk <= 0) chunk = lbm::kTQChunk;
  if (lag <= 0) lag = lbm::kTQLag;
  const int TS = (int)std::min<long long>(chunk, (long long)nx * ny);
  std::vector<int> nb, tk;
  const int nch = queue_schedule(nx, ny, nz, TS, lag, nb, tk);
  if (nch < 0) return -1;
  if (nbr) std::copy(nb.begin(), nb.end(), nbr);
  if (tasks) std::copy(tk.begin(), tk.end(), tasks);
  return nch;
}

int64_t lbm_revolve_steps(int64_t n, int snapshots) {
  if (n < 1 || snapshots < 0) return -1;
  if (snapshots == 0 || snapshots >= n) return n - 1;
  return revolve_count(n, snapshots);
}

lbm_status lbm_set_adjoint_memory(lbm_ctx* c, int snapshots) {
  if (!c) return LBM_ERR_ARG;
  if (snapshots < 0) return fail(c, LBM_ERR_ARG, "snapshots must be >= 0");
  c->adj_snaps = snapshots;
  return LBM_OK;
}

lbm_status lbm_test_adjoint_overlap(lbm_ctx* c, int on) {
  if (!c) return LBM_ERR_ARG;
  if (on != 0 && on != 1) return fail(c, LBM_ERR_ARG, "on must be 0 or 1");
  c->adj_overlap = on == 1;
  return LBM_OK;
}

lbm_status lbm_adjoint(lbm_ctx* c, const double* drho, double* dkij, double* dgamma, double* drho0) {
  if (!c || !drho) return c ? fail(c, LBM_ERR_ARG, "drho is NULL") : LBM_ERR_ARG;
  if (c->rec_t0 < 0 || c->rec_t0 + c->rec_n != c->t)
    return fail(c, LBM_ERR_ARG, "no recording ends at the current step (call lbm_record)");
  const lbm::AdjFns* A = lbm::adj_fns(c->Q, c->nc, c->precision, c->collision == LBM_MRT);
  const int64_t N = c->P.N;
  const int nc = c->nc, Q = c->Q, K = c->ck_every;
  const size_t sbytes = lbm_state_bytes(c), lbytes = (size_t)nc * Q * N * A->real_bytes;
  const unsigned nblk = A->rows(c->P);  // rows of the partial sums: one per block of any pass
  // revolve-style reversal inside each segment with S state slots when S < K; otherwise every
  // state of a segment is recomputed once and kept (K slots)
  const int S = (c->adj_snaps > 0 && c->adj_snaps < K) ? c->adj_snaps : 0;
  std::vector<void*> snaps((size_t)(S > 0 ? S + 2 : K), nullptr);
  // lam = X + rbB: X (la / lb, swapped every reverse step) and rbB per site and component.
  // Fbuf and rhob carry Fbar and the densities from pass A to pass B; pass A writes the pair
  // the following pass B does not read (index fc ^ 1, fc flipping with every pass A).
  void *la = nullptr, *lb = nullptr, *rbB = nullptr, *psis = nullptr;
  void *Fbuf[2] = {nullptr, nullptr}, *rhob[2] = {nullptr, nullptr};
  double *gpart = nullptr, *kpart = nullptr, *dd = nullptr;
  int* st_s = nullptr;
  long long* t_s = nullptr;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  // each set of state slots is one allocation, slots 256-byte aligned
  const size_t sstride = (sbytes + 255) & ~(size_t)255;
  void* slab = nullptr;
  alloc(&slab, snaps.size() * sstride);
  if (e == cudaSuccess)
    for (size_t i = 0; i < snaps.size(); ++i) snaps[i] = (char*)slab + i * sstride;
  // psi of every state of a segment, computed once by the replay and read by the reverse steps
  const size_t pbytes = (size_t)N * c->ops->psi_bytes;
  // revolve: plane 0 for the advances, planes 1 and 2 for psi of the last two reversed states
  alloc(&psis, (size_t)(S > 0 ? 3 : K) * pbytes);
  alloc(&la, lbytes);
  alloc(&lb, lbytes);
  for (int i = 0; i < 2; ++i) {
    alloc(&Fbuf[i], (size_t)3 * N * A->real_bytes);
    alloc(&rhob[i], (size_t)nc * N * A->real_bytes);
  }
  alloc(&rbB, (size_t)nc * N * A->real_bytes);
  alloc((void**)&gpart, (size_t)nblk * nc * sizeof(double));
  alloc((void**)&kpart, (size_t)nblk * nc * nc * sizeof(double));
  alloc((void**)&dd, (size_t)nc * N * sizeof(double));
  alloc((void**)&st_s, sizeof(int));
  alloc((void**)&t_s, sizeof(long long));
  // Full storage: a second set of segment slots lets the replay of segment k - 1 run on a
  // stream of its own while segment k is reversed (at small sizes both are latency-bound, and
  // they share no buffer). Without room for it the two alternate on one stream.
  std::vector<void*> snaps2;
  void *slab2 = nullptr, *psis2 = nullptr;
  cudaStream_t rs = c->stream;
  cudaEvent_t ev_rep[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
  bool two = false;
  if (e == cudaSuccess && S == 0 && c->ckpt.size() > 1 && c->adj_overlap) {
    bool ok = true;
    ok = cudaMalloc(&slab2, (size_t)K * sstride) == cudaSuccess;
    if (ok)
      for (int i = 0; i < K; ++i) snaps2.push_back((char*)slab2 + (size_t)i * sstride);
    ok = ok && cudaMalloc(&psis2, (size_t)K * pbytes) == cudaSuccess;
    cudaStream_t own = nullptr;
    ok = ok && cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) == cudaSuccess;
    if (own) rs = own;
    for (int i = 0; i < 2; ++i) {
      ok = ok && cudaEventCreateWithFlags(&ev_rep[i], cudaEventDisableTiming) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&ev_rev[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {  // not an error: the serial order needs none of it
      cudaGetLastError();
      cudaFree(slab2);
      slab2 = nullptr;
      snaps2.clear();
      cudaFree(psis2);
      psis2 = nullptr;
      if (own) cudaStreamDestroy(own);
      rs = c->stream;
      for (int i = 0; i < 2; ++i) {
        if (ev_rep[i]) cudaEventDestroy(ev_rep[i]);
        if (ev_rev[i]) cudaEventDestroy(ev_rev[i]);
        ev_rep[i] = ev_rev[i] = nullptr;
      }
    }
    two = ok;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(gpart, 0, (size_t)nblk * nc * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(kpart, 0, (size_t)nblk * nc * nc * sizeof(double), c->stream);
  for (int i = 0; i < 2; ++i)
    if (e == cudaSuccess) e = cudaMemsetAsync(Fbuf[i], 0, (size_t)3 * N * A->real_bytes, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(st_s, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dd, drho, (size_t)nc * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    A->seed(c->P, dd, la, rbB, c->stream);
    e = cudaGetLastError();
  }
  // One segment after its checkpoint is copied to slot 0 of a slot set: the replay recomputes
  // states t_k + 1 .. t_k + len - 1, each step reading slot i - 1 and writing slot i, keeping
  // psi of every state; the reverse steps then read them and swap la and lb once each.
  void** set_snaps[2] = {snaps.data(), two ? snaps2.data() : snaps.data()};
  void* set_psis[2] = {psis, two ? psis2 : psis};
  auto psi_in = [&](int set, int i) { return (void*)((char*)set_psis[set] + (size_t)i * pbytes); };
  auto replay = [&](int64_t tk, int len, int set) {
    void** sn = set_snaps[set];
    cudaError_t r = cudaSuccess;
    for (int i = 1; i < len && r == cudaSuccess; ++i) {
      const int parity = (int)((tk + i - 1) & 1);
      c->ops->psi(c->P, sn[i - 1], psi_in(set, i - 1), st_s, parity, rs);
      c->ops->collide_oop(c->P, sn[i - 1], sn[i], psi_in(set, i - 1), st_s, t_s, parity, rs);
      r = cudaGetLastError();
    }
    if (r == cudaSuccess) {
      c->ops->psi(c->P, sn[len - 1], psi_in(set, len - 1), st_s, (int)((tk + len - 1) & 1), rs);
      r = cudaGetLastError();
    }
    return r;
  };
  // The reverse sweep of a segment: pass A of its last step (lam(t + 1) from the seed or the
  // previous segment's closing pass B), then pass B + pass A per step down to the first, then
  // the closing pass B of the first state. fc: la == la0 ? 0 : 1 at the start.
  auto reverse = [&](int64_t tk, int len, int set, void* la_, void* lb_, int fc) {
    void** sn = set_snaps[set];
    int i = len - 1;
    A->pass_a(c->P, sn[i], psi_in(set, i), la_, rbB, lb_, Fbuf[fc ^ 1], rhob[fc ^ 1], (int)((tk + i) & 1), gpart,
              c->stream);
    std::swap(la_, lb_);
    fc ^= 1;
    cudaError_t r = cudaGetLastError();
    for (i = len - 2; i >= 0 && r == cudaSuccess; --i) {
      A->pass_ab(c->P, sn[i], psi_in(set, i), psi_in(set, i + 1), la_, lb_, Fbuf[fc], Fbuf[fc ^ 1], rhob[fc],
                 rhob[fc ^ 1], rbB, (int)((tk + i) & 1), gpart, kpart, c->stream);
      std::swap(la_, lb_);
      fc ^= 1;
      r = cudaGetLastError();
    }
    if (r == cudaSuccess) {
      A->pass_b(c->P, psi_in(set, 0), Fbuf[fc], rhob[fc], rbB, kpart, c->stream);
      r = cudaGetLastError();
    }
    return r;
  };
  // Revolve-style reversal of steps [t0, t0 + n) from the state at t0 in `base`, with the free
  // slots snaps[0 .. s) and the scratch buffers snaps[S], snaps[S + 1] (out-of-place steps
  // alternate between them). One step back needs its state and psi: psi into psis, pass A, pass B.
  // Recomputed states are bit-identical to the recorded ones, so the gradients equal those of
  // the full-storage schedule bit for bit.
  auto advance = [&](int64_t t0, const void* from, int64_t m, void* to) {
    // m >= 1 out-of-place steps from `from` (state t0); the last lands in `to`
    cudaError_t r = cudaSuccess;
    const void* cur = from;
    void* scratch[2] = {snaps[S], snaps[S + 1]};
    for (int64_t i = 0; i < m && r == cudaSuccess; ++i) {
      void* nxt = i == m - 1 ? to : scratch[(m - 1 - i) & 1];
      const int parity = (int)((t0 + i) & 1);
      c->ops->psi(c->P, cur, psis, st_s, parity, c->stream);
      c->ops->collide_oop(c->P, cur, nxt, psis, st_s, t_s, parity, c->stream);
      r = cudaGetLastError();
      cur = nxt;
    }
    return r;
  };
  void* const la0 = la;  // which X buffer is current: la == la0 after an even number of passes A
  // One step back, the same launches as the full-storage sweep: psi of its state into the plane
  // of its parity, pass A alone for a segment's first reversed step, else pass B of the step
  // after it (whose psi is still in the other plane) with pass A; the segment's closing pass B
  // follows its revolve.
  auto psi_rev = [&](int64_t t) { return (void*)((char*)psis + (size_t)(1 + (t & 1)) * pbytes); };
  bool b_pending = false;
  auto back_step = [&](int64_t t, const void* state) {
    const int parity = (int)(t & 1);
    const int fc = la == la0 ? 0 : 1;
    c->ops->psi(c->P, state, psi_rev(t), st_s, parity, c->stream);
    if (!b_pending)
      A->pass_a(c->P, state, psi_rev(t), la, rbB, lb, Fbuf[fc ^ 1], rhob[fc ^ 1], parity, gpart, c->stream);
    else
      A->pass_ab(c->P, state, psi_rev(t), psi_rev(t + 1), la, lb, Fbuf[fc], Fbuf[fc ^ 1], rhob[fc], rhob[fc ^ 1], rbB,
                 parity, gpart, kpart, c->stream);
    b_pending = true;
    std::swap(la, lb);
    return cudaGetLastError();
  };
  std::function<cudaError_t(int64_t, int64_t, const void*, int)> revolve = [&](int64_t t0, int64_t n,
                                                                                const void* base, int s_) {
    if (n == 1) return back_step(t0, base);
    if (s_ == 0) {  // no slot left: recompute each state from the base, last first
      cudaError_t r = cudaSuccess;
      for (int64_t i = n - 1; i >= 0 && r == cudaSuccess; --i) {
        if (i == 0) {
          r = back_step(t0, base);
        } else {
          r = advance(t0, base, i, snaps[S]);
          if (r == cudaSuccess) r = back_step(t0 + i, snaps[S]);
        }
      }
      return r;
    }
    const int64_t m = binomial_split(n, s_);
    void* slot = snaps[s_ - 1];
    cudaError_t r = advance(t0, base, m, slot);
    if (r == cudaSuccess) r = revolve(t0 + m, n - m, slot, s_ - 1);
    if (r == cudaSuccess) r = revolve(t0, m, base, s_);
    return r;
  };
  // Full segments repeat the same launches: the replay is captured as a graph per (parity of
  // t_k, slot set), the reverse sweep per (parity of t_k, which buffer is la, slot set), and
  // replayed; a failed capture falls back to direct launches.
  bool capture_ok = true;
  auto captured = [&](cudaGraphExec_t& g, cudaStream_t st, const std::function<cudaError_t()>& body) {
    if (!g && capture_ok) {
      cudaGraph_t graph = nullptr;
      capture_ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (capture_ok) {
        const cudaError_t r = body();
        capture_ok = cudaStreamEndCapture(st, &graph) == cudaSuccess && r == cudaSuccess && graph &&
                     cudaGraphInstantiate(&g, graph, 0) == cudaSuccess;
        if (graph) cudaGraphDestroy(graph);
      }
      if (!capture_ok) {
        g = nullptr;
        cudaGetLastError();
      }
    }
    return g ? cudaGraphLaunch(g, st) : body();
  };
  cudaGraphExec_t g_rep[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t g_rev[2][2][2] = {{{nullptr, nullptr}, {nullptr, nullptr}}, {{nullptr, nullptr}, {nullptr, nullptr}}};
  const int nseg = (int)c->ckpt.size();
  auto seg_t = [&](int k) { return c->rec_t0 + (int64_t)k * K; };
  auto seg_len = [&](int k) { return (int)std::min<int64_t>(K, c->rec_t0 + c->rec_n - seg_t(k)); };
  auto set_of = [&](int k) { return two ? (k & 1) : 0; };
  // Replay of segment k on rs, after the reverse sweep that last read its slot set.
  auto run_replay = [&](int k) {
    const int set = set_of(k), len = seg_len(k);
    const int64_t tk = seg_t(k);
    cudaError_t r = two ? cudaStreamWaitEvent(rs, ev_rev[set], 0) : cudaSuccess;
    if (r == cudaSuccess) r = cudaMemcpyAsync(set_snaps[set][0], c->ckpt[k], sbytes, cudaMemcpyDeviceToDevice, rs);
    if (r != cudaSuccess) return r;
    auto body = [&]() { return replay(tk, len, set); };
    r = (len == K && K > 1) ? captured(g_rep[tk & 1][set], rs, body) : body();
    if (r == cudaSuccess && two) r = cudaEventRecord(ev_rep[set], rs);
    return r;
  };
  // Reverse sweep of segment k on the context's stream, after its replay.
  auto run_reverse = [&](int k) {
    const int set = set_of(k), len = seg_len(k);
    const int64_t tk = seg_t(k);
    cudaError_t r = two ? cudaStreamWaitEvent(c->stream, ev_rep[set], 0) : cudaSuccess;
    if (r != cudaSuccess) return r;
    void *a = la, *b = lb;
    const int fc = la == la0 ? 0 : 1;
    auto body = [&]() { return reverse(tk, len, set, a, b, fc); };
    r = (len == K && K > 1) ? captured(g_rev[tk & 1][la == la0 ? 0 : 1][set], c->stream, body) : body();
    if (len & 1) std::swap(la, lb);
    if (r == cudaSuccess && two) r = cudaEventRecord(ev_rev[set], c->stream);
    return r;
  };
  if (e == cudaSuccess && S == 0 && nseg > 0) e = run_replay(nseg - 1);
  for (int k = nseg - 1; k >= 0 && e == cudaSuccess; --k) {
    if (S > 0) {  // the recorded checkpoint is read, never written
      e = revolve(seg_t(k), seg_len(k), c->ckpt[k], S);
      if (e == cudaSuccess) {
        const int fc = la == la0 ? 0 : 1;
        A->pass_b(c->P, psi_rev(seg_t(k)), Fbuf[fc], rhob[fc], rbB, kpart, c->stream);
        b_pending = false;
        e = cudaGetLastError();
      }
      continue;
    }
    if (two && k >= 1) e = run_replay(k - 1);  // runs beside the reverse sweep of segment k
    if (e == cudaSuccess) e = run_reverse(k);
    if (e == cudaSuccess && !two && k >= 1) e = run_replay(k - 1);
  }
  if (two) {
    const cudaError_t r = cudaStreamSynchronize(rs);
    if (e == cudaSuccess) e = r;
  }
  for (auto& row : g_rep)
    for (auto& g : row)
      if (g) cudaGraphExecDestroy(g);
  for (auto& pl : g_rev)
    for (auto& row : pl)
      for (auto& g : row)
        if (g) cudaGraphExecDestroy(g);
  if (e == cudaSuccess && drho0) {
    A->init_grad(c->P, la, rbB, dd, c->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(drho0, dd, (size_t)nc * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  }
  std::vector<double> hg((size_t)nblk * nc), hk((size_t)nblk * nc * nc);
  int hst = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hg.data(), gpart, hg.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hk.data(), kpart, hk.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, st_s, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(slab);
  cudaFree(slab2);
  cudaFree(psis);
  cudaFree(psis2);
  if (two) {
    cudaStreamDestroy(rs);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(ev_rep[i]);
      cudaEventDestroy(ev_rev[i]);
    }
  }
  cudaFree(la);
  cudaFree(lb);
  for (int i = 0; i < 2; ++i) {
    cudaFree(Fbuf[i]);
    cudaFree(rhob[i]);
  }
  cudaFree(rbB);
  cudaFree(gpart);
  cudaFree(kpart);
  cudaFree(dd);
  cudaFree(st_s);
  cudaFree(t_s);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_adjoint");
  if (hst) return fail(c, LBM_ERR_PSI_DOMAIN, "recomputed forward step left the EOS domain");
  if (dgamma)
    for (int i = 0; i < nc; ++i) {
      double acc = 0;
      for (unsigned bb = 0; bb < nblk; ++bb) acc += hg[(size_t)bb * nc + i];
      dgamma[i] = acc;
    }
  if (dkij)
    for (int i = 0; i < nc * nc; ++i) {
      double acc = 0;
      for (unsigned bb = 0; bb < nblk; ++bb) acc += hk[(size_t)bb * nc * nc + i];
      dkij[i] = acc;
    }
  return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

lbm_status lbm_scale_to_lattice(int nc, const lbm_component* phys, double T_phys, double p_phys,
                                lbm_component* out, double* T_lb, double* p_lb) {
  if (nc < 1 || nc > 4 || !phys || !out || !(phys[0].Tc > 0) || !(phys[0].pc > 0) || !(phys[0].M > 0))
    return LBM_ERR_ARG;
  const double a1 = 2.0 / 49.0, b1 = 2.0 / 21.0;
  const double Tc1 = (kOmegaB / kOmegaA) * (a1 / b1);
  const double pc1 = kOmegaB * Tc1 / b1;
  const double ts = Tc1 / phys[0].Tc, ps = pc1 / phys[0].pc;
  for (int i = 0; i < nc; ++i) {
    if (!(phys[i].Tc > 0) || !(phys[i].pc > 0) || !(phys[i].M > 0)) return LBM_ERR_ARG;
    out[i].Tc = phys[i].Tc * ts;
    out[i].pc = phys[i].pc * ps;
    out[i].omega = phys[i].omega;
    out[i].M = phys[i].M / phys[0].M;
  }
  if (T_lb) *T_lb = T_phys * ts;
  if (p_lb) *p_lb = p_phys * ps;
  return LBM_OK;
}

}  // extern "C"
