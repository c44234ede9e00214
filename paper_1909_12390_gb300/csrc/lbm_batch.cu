// Batched lattices: many small independent D2Q9 cases (their own grid, temperature, feed,
// volatility coefficients) advanced together. Each block owns one case for a whole chunk of
// steps: the case's populations and pseudo-potential are loaded into shared memory once, every
// step runs out of shared memory with block barriers between the pseudo-potential pass and the
// collide-stream pass, and the state is written back at the end of the chunk. Cases are grouped
// by size; each size class is one launch on its own stream with a block size chosen by a small
// autotuner, and the fork-join of the class launches is captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_kernels.cuh"

namespace lbm {

struct BatchCase {
  Params P;
  int64_t f_off;     // element offset of the case's populations in the batch buffer
  int64_t site_off;  // site offset of the case (pseudo-potential buffer, fields)
};

// One step of one case held by this block: psi of every site, barrier, collide and stream.
// Returns the status bits of the psi pass (uniform over the block).
template <int Q, int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ int batch_step(const Params& P, typename Prec::S* f, typename Prec::PsiT* psi) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  const uint32_t N = P.N32;
  int err = 0;
  for (uint32_t idx = threadIdx.x; idx < N; idx += blockDim.x) {
    Site s;
    s.set(P, idx);
    typename Prec::PsiT v;
    err |= site_psi<Q, NC, Prec, PAR>(P, f, s, v);
    psi[idx] = v;
  }
  err = __syncthreads_or(err);
  if (err) return err;
  for (uint32_t idx = threadIdx.x; idx < N; idx += blockDim.x) {
    Site s;
    s.set(P, idx);
    R pn[Q];
    pn[0] = (R)psi[idx];
#pragma unroll
    for (int a = 1; a < Q; ++a) pn[a] = (R)psi[s.nb(P, L::e(a, 0), L::e(a, 1), L::e(a, 2))];
    site_collide<Q, NC, Prec, MRT, PAR, 0>(P, f, s, pn);  // f may point into shared memory
  }
  __syncthreads();
  return 0;
}

template <int Q, int NC, class Prec, int MRT>
__global__ void k_batch(const BatchCase* __restrict__ cases, const int* __restrict__ order, typename Prec::S* f_all,
                        typename Prec::PsiT* psi_all, int* case_status, long long* case_t, int nsteps, int use_smem) {
  using S = typename Prec::S;
  using PsiT = typename Prec::PsiT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Params P;
  __shared__ int64_t foff, soff;
  const int ci = order[blockIdx.x];
  if (threadIdx.x == 0) {
    P = cases[ci].P;
    foff = cases[ci].f_off;
    soff = cases[ci].site_off;
  }
  __syncthreads();
  const int64_t N = P.N;
  const int64_t nf = (int64_t)NC * Q * N;
  const size_t fbytes = ((size_t)nf * sizeof(S) + 15) & ~(size_t)15;
  S* f = use_smem ? (S*)smem : f_all + foff;
  PsiT* psi = use_smem ? (PsiT*)(smem + fbytes) : psi_all + soff;
  if (use_smem)
    for (int64_t i = threadIdx.x; i < nf; i += blockDim.x) f[i] = f_all[foff + i];
  __syncthreads();
  const long long t0 = case_t[ci];
  int st = case_status[ci];
  int done = 0;
  for (int k = 0; k < nsteps && st == 0; ++k) {
    const int err = ((t0 + k) & 1) ? batch_step<Q, NC, Prec, MRT, 1>(P, f, psi)
                                   : batch_step<Q, NC, Prec, MRT, 0>(P, f, psi);
    if (err) {
      st = err;
      break;
    }
    ++done;
  }
  if (use_smem)
    for (int64_t i = threadIdx.x; i < nf; i += blockDim.x) f_all[foff + i] = f[i];
  if (threadIdx.x == 0) {
    case_status[ci] = st;
    case_t[ci] = t0 + done;
  }
}

struct BatchFns {
  cudaError_t (*launch)(const BatchCase*, const int*, void*, void*, int*, long long*, int nsteps, int use_smem,
                        int nblocks, int threads, size_t smem, cudaStream_t);
  cudaError_t (*attrs)(cudaFuncAttributes*);
  cudaError_t (*set_smem)(int bytes);
  int store_bytes, psi_bytes;
};

template <int Q, int NC, class Prec, int MRT>
struct BatchLaunch {
  static cudaError_t launch(const BatchCase* cs, const int* order, void* f, void* psi, int* st, long long* t,
                            int nsteps, int use_smem, int nblocks, int threads, size_t smem, cudaStream_t s) {
    k_batch<Q, NC, Prec, MRT><<<nblocks, threads, smem, s>>>(cs, order, (typename Prec::S*)f,
                                                             (typename Prec::PsiT*)psi, st, t, nsteps, use_smem);
    return cudaGetLastError();
  }
  static cudaError_t attrs(cudaFuncAttributes* a) { return cudaFuncGetAttributes(a, k_batch<Q, NC, Prec, MRT>); }
  static cudaError_t set_smem(int bytes) {
    return cudaFuncSetAttribute(k_batch<Q, NC, Prec, MRT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  static const BatchFns* table() {
    static const BatchFns t = {launch, attrs, set_smem, (int)sizeof(typename Prec::S),
                               (int)sizeof(typename Prec::PsiT)};
    return &t;
  }
};

template <class Prec, int MRT>
const BatchFns* batch_nc(int nc) {
  switch (nc) {
    case 1: return BatchLaunch<9, 1, Prec, MRT>::table();
    case 2: return BatchLaunch<9, 2, Prec, MRT>::table();
    case 3: return BatchLaunch<9, 3, Prec, MRT>::table();
    case 4: return BatchLaunch<9, 4, Prec, MRT>::table();
  }
  return nullptr;
}

const BatchFns* batch_fns(int nc, int precision, int collision) {
  if (precision == LBM_FP64) return collision ? batch_nc<PrecF64, 1>(nc) : batch_nc<PrecF64, 0>(nc);
  return collision ? batch_nc<PrecF32S, 1>(nc) : batch_nc<PrecF32S, 0>(nc);
}

}  // namespace lbm

namespace {

const int kChunk = 100;  // steps per class launch inside the captured graph

struct SizeClass {
  int64_t N = 0;
  std::vector<int> cases;
  int* d_order = nullptr;
  int threads = 256;
  int use_smem = 0;
  size_t smem = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

thread_local std::string g_batch_create_error;

}  // namespace

struct lbm_batch {
  int ncase = 0, nc = 0, precision = 0, collision = 0;
  std::vector<lbm::BatchCase> cases;
  std::vector<bool> ref_given;
  const lbm::Ops* ops = nullptr;
  const lbm::BatchFns* fns = nullptr;
  lbm::BatchCase* d_cases = nullptr;
  void* f = nullptr;
  void* psi = nullptr;
  int* d_status = nullptr;
  long long* d_t = nullptr;
  double* scratch = nullptr;
  int64_t n_max = 0, sites = 0, pops = 0;
  std::vector<SizeClass> classes;
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  int64_t t = 0;
  std::string err;
  std::string tune_report;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b)
    b->err = buf;
  else
    g_batch_create_error = buf;
  return st;
}

#define BCK(b, call)                                                                                     \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA, "%s: %s", #call,     \
                   cudaGetErrorString(e_));                                                              \
  } while (0)

// Launches every size class for nsteps steps, forked from and joined back into b->stream.
cudaError_t launch_classes(lbm_batch* b, int nsteps) {
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  for (auto& c : b->classes) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c.stream, b->fork, 0);
    if (e == cudaSuccess)
      e = b->fns->launch(b->d_cases, c.d_order, b->f, b->psi, b->d_status, b->d_t, nsteps, c.use_smem,
                         (int)c.cases.size(), c.threads, c.smem, c.stream);
    if (e == cudaSuccess) e = cudaEventRecord(c.done, c.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, c.done, 0);
  }
  return e;
}

void drop_graph(lbm_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

bool build_graph(lbm_batch* b) {
  if (b->graph) return true;
  if (b->graph_failed) return false;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    b->graph_failed = true;
    return false;
  }
  cudaError_t e = launch_classes(b, kChunk);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess || !g || cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    b->graph = nullptr;
    b->graph_failed = true;
    return false;
  }
  cudaGraphDestroy(g);
  return true;
}

// Shared-memory bytes of one case of N sites, 0 if it does not fit.
size_t smem_need(const lbm_batch* b, int64_t N, int smem_max) {
  const size_t fb = ((size_t)b->nc * 9 * N * b->fns->store_bytes + 15) & ~(size_t)15;
  const size_t need = fb + (size_t)N * b->fns->psi_bytes;
  return need <= (size_t)smem_max ? need : 0;
}

lbm_status upload_cases(lbm_batch* b) {
  BCK(b, cudaMemcpyAsync(b->d_cases, b->cases.data(), b->cases.size() * sizeof(lbm::BatchCase),
                         cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int ncase, const lbm_grid* grids, int nc, const lbm_component* comps,
                            const lbm_eos* eos, const double* tau, lbm_batch** out) {
  g_batch_create_error.clear();
  if (!out) return bfail(nullptr, LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (ncase < 1 || !grids || !comps || !eos || !tau) return bfail(nullptr, LBM_ERR_ARG, "empty batch or NULL arrays");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(nullptr, LBM_ERR_OOM, "host allocation failed");
  b->ncase = ncase;
  b->nc = nc;
  b->precision = eos[0].precision;
  b->collision = eos[0].collision;
  b->cases.resize(ncase);
  b->ref_given.resize(ncase);
  int64_t fo = 0, so = 0;
  for (int i = 0; i < ncase; ++i) {
    if (grids[i].lattice != LBM_D2Q9) {
      delete b;
      return bfail(nullptr, LBM_ERR_ARG, "case %d: batched cases must be D2Q9", i);
    }
    if (eos[i].precision != b->precision || eos[i].collision != b->collision) {
      delete b;
      return bfail(nullptr, LBM_ERR_ARG, "case %d: every case needs the same precision and collision", i);
    }
    const lbm::Ops* ops = nullptr;
    std::string why;
    lbm_status st = lbm::make_params(&grids[i], nc, comps + (size_t)i * nc, &eos[i], tau[i], &b->cases[i].P, &ops, &why);
    if (st != LBM_OK) {
      delete b;
      return bfail(nullptr, st, "case %d: %s", i, why.c_str());
    }
    b->ops = ops;
    b->ref_given[i] = eos[i].rho_ref != nullptr;
    const int64_t N = b->cases[i].P.N;
    b->cases[i].f_off = fo;
    b->cases[i].site_off = so;
    fo += (int64_t)nc * 9 * N;
    so += N;
    b->n_max = std::max(b->n_max, N);
  }
  b->sites = so;
  b->pops = fo;
  b->fns = lbm::batch_fns(nc, b->precision, b->collision);
  int dev = 0, smem_max = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_cases, (size_t)ncase * sizeof(lbm::BatchCase));
  if (e == cudaSuccess) e = cudaMalloc(&b->f, (size_t)fo * b->fns->store_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->psi, (size_t)so * b->fns->psi_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, (size_t)ncase * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_t, (size_t)ncase * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, (size_t)ncase * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_t, 0, (size_t)ncase * sizeof(long long));
  // size classes, largest first
  std::map<int64_t, std::vector<int>, std::greater<int64_t>> by_size;
  for (int i = 0; i < ncase; ++i) by_size[b->cases[i].P.N].push_back(i);
  const int fit_max = smem_max - 1024;  // leave room for the static shared parameters
  for (auto& kv : by_size) {
    if (e != cudaSuccess) break;
    SizeClass c;
    c.N = kv.first;
    c.cases = kv.second;
    c.smem = smem_need(b, c.N, fit_max);
    c.use_smem = c.smem > 0;
    e = cudaMalloc(&c.d_order, c.cases.size() * sizeof(int));
    if (e == cudaSuccess)
      e = cudaMemcpy(c.d_order, c.cases.data(), c.cases.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
    b->classes.push_back(c);
  }
  size_t smem_hi = 0;
  for (auto& c : b->classes) smem_hi = std::max(smem_hi, c.smem);
  if (e == cudaSuccess && smem_hi > 0) e = b->fns->set_smem((int)smem_hi);
  if (e != cudaSuccess) {
    lbm_status st = e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    bfail(nullptr, st, "lbm_batch_create: %s", cudaGetErrorString(e));
    lbm_batch_destroy(b);
    return st;
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (auto& c : b->classes) {
    if (c.stream) cudaStreamSynchronize(c.stream);
    cudaFree(c.d_order);
    if (c.stream) cudaStreamDestroy(c.stream);
    if (c.done) cudaEventDestroy(c.done);
  }
  cudaFree(b->d_cases);
  cudaFree(b->f);
  cudaFree(b->psi);
  cudaFree(b->d_status);
  cudaFree(b->d_t);
  cudaFree(b->scratch);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

lbm_status lbm_batch_init(lbm_batch* b, const double* rho, const double* u) {
  if (!b || !rho) return b ? bfail(b, LBM_ERR_ARG, "rho is NULL") : LBM_ERR_ARG;
  const int nc = b->nc;
  for (int i = 0; i < b->ncase; ++i) {
    lbm::BatchCase& c = b->cases[i];
    const int64_t N = c.P.N;
    const double* r = rho + (size_t)c.site_off * nc;
    for (int s = 0; s < nc; ++s) {
      double m = r[s * N];
      for (int64_t k = 0; k < N; ++k) {
        const double v = r[s * N + k];
        if (!(v > 0) || !std::isfinite(v))
          return bfail(b, LBM_ERR_ARG, "case %d: rho must be finite and > 0", i);
        m = std::min(m, v);
      }
      if (b->precision == LBM_FP32_SHIFTED && !b->ref_given[i]) c.P.rho_ref[s] = m;
    }
    lbm::finalize_params(c.P);
  }
  if (!b->scratch) BCK(b, cudaMalloc(&b->scratch, (size_t)(nc + 5) * b->n_max * sizeof(double)));
  for (int i = 0; i < b->ncase; ++i) {
    const lbm::BatchCase& c = b->cases[i];
    const int64_t N = c.P.N;
    BCK(b, cudaMemcpyAsync(b->scratch, rho + (size_t)c.site_off * nc, (size_t)nc * N * sizeof(double),
                           cudaMemcpyHostToDevice, b->stream));
    if (u)
      BCK(b, cudaMemcpyAsync(b->scratch + (size_t)nc * N, u + (size_t)c.site_off * 3, (size_t)3 * N * sizeof(double),
                             cudaMemcpyHostToDevice, b->stream));
    b->ops->init(c.P, (char*)b->f + (size_t)c.f_off * b->fns->store_bytes, b->scratch,
                 u ? b->scratch + (size_t)nc * N : nullptr, b->stream);
    BCK(b, cudaGetLastError());
  }
  BCK(b, cudaMemsetAsync(b->d_status, 0, (size_t)b->ncase * sizeof(int), b->stream));
  BCK(b, cudaMemsetAsync(b->d_t, 0, (size_t)b->ncase * sizeof(long long), b->stream));
  drop_graph(b);
  lbm_status st = upload_cases(b);
  if (st != LBM_OK) return st;
  b->t = 0;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
  if (!b) return LBM_ERR_ARG;
  if (n < 0) return bfail(b, LBM_ERR_ARG, "n must be >= 0");
  int64_t left = n;
  while (left >= kChunk && build_graph(b)) {
    BCK(b, cudaGraphLaunch(b->graph, b->stream));
    left -= kChunk;
  }
  while (left > 0) {
    const int k = (int)std::min<int64_t>(left, 1 << 20);
    BCK(b, launch_classes(b, k));
    left -= k;
  }
  BCK(b, cudaStreamSynchronize(b->stream));
  std::vector<int> st(b->ncase);
  BCK(b, cudaMemcpy(st.data(), b->d_status, (size_t)b->ncase * sizeof(int), cudaMemcpyDeviceToHost));
  b->t += n;
  for (int i = 0; i < b->ncase; ++i) {
    if (st[i] & lbm::ST_NONFINITE) return bfail(b, LBM_ERR_NONFINITE, "case %d: non-finite density or psi^2", i);
    if (st[i] & lbm::ST_PSI_DOMAIN) return bfail(b, LBM_ERR_PSI_DOMAIN, "case %d: psi^2 < 0 or b_m n >= 1", i);
  }
  return LBM_OK;
}

lbm_status lbm_batch_case_status(lbm_batch* b, int* status, int64_t* t) {
  if (!b) return LBM_ERR_ARG;
  std::vector<int> st(b->ncase);
  std::vector<long long> tt(b->ncase);
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, cudaMemcpy(st.data(), b->d_status, (size_t)b->ncase * sizeof(int), cudaMemcpyDeviceToHost));
  BCK(b, cudaMemcpy(tt.data(), b->d_t, (size_t)b->ncase * sizeof(long long), cudaMemcpyDeviceToHost));
  for (int i = 0; i < b->ncase; ++i) {
    if (status)
      status[i] = st[i] == 0 ? LBM_OK : ((st[i] & lbm::ST_NONFINITE) ? LBM_ERR_NONFINITE : LBM_ERR_PSI_DOMAIN);
    if (t) t[i] = tt[i];
  }
  return LBM_OK;
}

// Per-case read-back through the single-lattice kernels on the case's slice of the buffers.
lbm_status lbm_batch_fields(lbm_batch* b, double* rho, double* u, double* p) {
  if (!b) return LBM_ERR_ARG;
  std::vector<long long> tt(b->ncase);
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, cudaMemcpy(tt.data(), b->d_t, (size_t)b->ncase * sizeof(long long), cudaMemcpyDeviceToHost));
  if (!b->scratch) BCK(b, cudaMalloc(&b->scratch, (size_t)(b->nc + 5) * b->n_max * sizeof(double)));
  int* st_dev = b->d_status;  // the psi pass only writes it on error, which lbm_batch_step reported already
  const int nc = b->nc;
  for (int i = 0; i < b->ncase; ++i) {
    const lbm::BatchCase& c = b->cases[i];
    const int64_t N = c.P.N;
    const int parity = (int)(tt[i] & 1);
    void* fi = (char*)b->f + (size_t)c.f_off * b->fns->store_bytes;
    void* pi = (char*)b->psi + (size_t)c.site_off * b->fns->psi_bytes;
    double* dr = b->scratch;
    double* du = dr + (size_t)nc * N;
    double* dp = du + (size_t)3 * N;
    double* dpsi = dp + N;
    int st0 = 0;
    BCK(b, cudaMemcpyAsync(&st0, st_dev + i, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
    if (st0) continue;  // a failed case keeps its last state; its fields are not computed
    // the two-kernel pseudo-potential pass reads the status word only as a stop flag
    b->ops->psi(c.P, fi, pi, st_dev + i, parity, b->stream);
    b->ops->fields(c.P, fi, pi, dr, du, dp, dpsi, parity, b->stream);
    BCK(b, cudaGetLastError());
    if (rho)
      BCK(b, cudaMemcpyAsync(rho + (size_t)c.site_off * nc, dr, (size_t)nc * N * sizeof(double),
                             cudaMemcpyDeviceToHost, b->stream));
    if (u)
      BCK(b, cudaMemcpyAsync(u + (size_t)c.site_off * 3, du, (size_t)3 * N * sizeof(double), cudaMemcpyDeviceToHost,
                             b->stream));
    if (p) BCK(b, cudaMemcpyAsync(p + c.site_off, dp, (size_t)N * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    BCK(b, cudaStreamSynchronize(b->stream));
  }
  return LBM_OK;
}

lbm_status lbm_batch_get_f(lbm_batch* b, int i, double* f) {
  if (!b || !f || i < 0 || i >= b->ncase) return b ? bfail(b, LBM_ERR_ARG, "bad case index or NULL f") : LBM_ERR_ARG;
  const lbm::BatchCase& c = b->cases[i];
  long long t = 0;
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, cudaMemcpy(&t, b->d_t + i, sizeof(long long), cudaMemcpyDeviceToHost));
  const size_t n = (size_t)b->nc * 9 * c.P.N;
  double* d = nullptr;  // read-back staging
  BCK(b, cudaMallocAsync(&d, n * sizeof(double), b->stream));
  b->ops->get_f(c.P, (char*)b->f + (size_t)c.f_off * b->fns->store_bytes, d, (int)(t & 1), b->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  cudaFreeAsync(d, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "lbm_batch_get_f: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Autotuner: for each size class, times trial_steps steps of every feasible block size on a
// scratch copy of the batch's populations and keeps the fastest.
lbm_status lbm_batch_tune(lbm_batch* b, int trial_steps) {
  if (!b || trial_steps < 1) return b ? bfail(b, LBM_ERR_ARG, "trial_steps must be >= 1") : LBM_ERR_ARG;
  cudaFuncAttributes fa{};
  BCK(b, b->fns->attrs(&fa));
  const int reg_threads = std::max(32, (65536 / std::max(fa.numRegs, 1)) / 32 * 32);
  const int max_threads = std::min(fa.maxThreadsPerBlock, reg_threads);
  void* f_save = nullptr;
  int* st_save = nullptr;
  long long* t_save = nullptr;
  const size_t fbytes = (size_t)b->pops * b->fns->store_bytes;
  BCK(b, cudaStreamSynchronize(b->stream));
  BCK(b, cudaMalloc(&f_save, fbytes));
  cudaError_t e = cudaMalloc(&st_save, (size_t)b->ncase * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&t_save, (size_t)b->ncase * sizeof(long long));
  if (e == cudaSuccess) e = cudaMemcpy(f_save, b->f, fbytes, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(st_save, b->d_status, (size_t)b->ncase * sizeof(int), cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t_save, b->d_t, (size_t)b->ncase * sizeof(long long), cudaMemcpyDeviceToDevice);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::string rep;
  for (auto& c : b->classes) {
    if (e != cudaSuccess) break;
    float best = 1e30f;
    int best_t = c.threads;
    for (int th = 64; th <= max_threads; th *= 2) {
      if (th > c.N * 2 && th > 64) break;
      e = cudaEventRecord(e0, c.stream);
      if (e == cudaSuccess)
        e = b->fns->launch(b->d_cases, c.d_order, b->f, b->psi, b->d_status, b->d_t, trial_steps, c.use_smem,
                           (int)c.cases.size(), th, c.smem, c.stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c.stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      if (ms < best) {
        best = ms;
        best_t = th;
      }
      // undo the trial steps
      e = cudaMemcpy(b->f, f_save, fbytes, cudaMemcpyDeviceToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(b->d_status, st_save, (size_t)b->ncase * sizeof(int), cudaMemcpyDeviceToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(b->d_t, t_save, (size_t)b->ncase * sizeof(long long), cudaMemcpyDeviceToDevice);
    }
    c.threads = best_t;
    char line[160];
    snprintf(line, sizeof line, "N=%lld cases=%zu smem=%d threads=%d %.3f ms/%d steps; ", (long long)c.N, c.cases.size(),
             c.use_smem, best_t, best, trial_steps);
    rep += line;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(f_save);
  cudaFree(st_save);
  cudaFree(t_save);
  drop_graph(b);
  b->graph_failed = false;
  b->tune_report = rep;
  if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "lbm_batch_tune: %s", cudaGetErrorString(e));
  return LBM_OK;
}

const char* lbm_batch_tune_report(const lbm_batch* b) { return b ? b->tune_report.c_str() : ""; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

int64_t lbm_batch_sites(const lbm_batch* b) { return b ? b->sites : -1; }

}  // extern "C"
