// Trailing fused D3Q19 step (k_trail3): one persistent cooperative launch per step, in which
// the pseudo-potential of the NEXT step trails the collision of this one.
//
// Step t needs psi(t) at every site before any collision, and psi(t) needs the densities of
// the state at t. Here psi(t) was finished by the launch of step t - 1 (or by a pseudo-potential
// pass before the first step), so the collisions of step t wait for nothing. CTA b owns the
// contiguous range [range[b], range[b+1]) of the flattened (y, x) index of a z plane and
// marches z = 0 .. nz-1; iteration k
//   1. collides and streams plane k of its range in place (psi(t) of the 18 neighbours from
//      the current buffer, read-only in this launch), then arrives on the plane's mbarrier;
//   2. the warp whose arrival completes the plane's mbarrier phase publishes the plane (a
//      release maximum on the CTA's progress flag);
//   3. computes psi(t + 1) of plane p = k - LAG of its range into the other buffer: the
//      densities of the state at t + 1 at a site are sums over slots written by the collisions
//      of planes p - 1 .. p + 1 of this CTA and of the CTAs owning neighbour sites, so the
//      stage first waits (bounded) for its own CTA's mbarrier of plane p + 1 and for the
//      neighbours' published progress >= p + 1. Those slots were written LAG - 1 .. LAG + 1
//      iterations earlier; with every CTA marching the same planes, the grid touches a few
//      planes meanwhile (15 MB each at 256^2 sites, three FP32 D3Q19 components), so the
//      re-reads come from L2.
// After the march the stages of planes nz - LAG .. nz - 1 and of plane 0 (which needs plane
// nz - 1) follow once every neighbour has finished. The result of a step is the same, bit for
// bit, as that of the two-kernel step: the collision is the same per-site code, and psi(t+1)
// of a site is site_psi over the same slots.
//
// Each site reads and writes only its own set of slots (AA pattern), so a site's collision
// never disturbs another site's populations; the only cross-site dependency is psi, and psi(t)
// is complete before the launch. The waits go only backwards in the march (a stage of plane p
// waits for collisions of planes <= p + 1 < k, published before the waiter's iteration), and
// the cooperative launch makes all CTAs co-resident, so the pipeline cannot deadlock; every
// wait is bounded anyway (kSpinLimit polls), after which the step reports a timeout.
// Errors of the psi(t + 1) stage (EOS domain, non-finite) are collected in A.pending and folded
// into the status word by the last CTA: step t completed, and the next step is the failing one.
#pragma once

namespace lbm {

#ifndef LBM_T3_THREADS
#define LBM_T3_THREADS 448
#endif
constexpr int kT3Threads = LBM_T3_THREADS;  // 14 warps, one site each of a 431-site range
// registers per thread: the warps of a CTA are spread over the SM's four sub-partitions, each
// with 16 K registers, so the busiest sub-partition (ceil(warps / 4) warps) bounds them: 128 for
// 14 warps, 168 for 12
#define LBM_T3_WPS ((LBM_T3_THREADS / 32 + 3) / 4)
#ifndef LBM_T3_MAXREG
#define LBM_T3_MAXREG (16384 / (LBM_T3_WPS * 32) / 8 * 8 > 255 ? 255 : 16384 / (LBM_T3_WPS * 32) / 8 * 8)
#endif
static_assert(kT3Threads % 32 == 0 && kT3Threads <= 1024, "trailing step block size");
// planes between a plane's collision and its psi(t + 1) stage
#ifndef LBM_T3_LAG
#define LBM_T3_LAG 4
#endif
constexpr int kT3Lag = LBM_T3_LAG;
static_assert(kT3Lag >= 2, "the psi stage of plane k - LAG needs plane k - LAG + 1 collided by the neighbours");
// population stores: 1 evict-first (st.global.cs), 2 write-back (st.global.wb, kept in L2 for the
// psi stage)
#ifndef LBM_T3_CS
#define LBM_T3_CS 2
#endif
constexpr int kT3Ring = 8;  // mbarriers, plane k on k % kT3Ring
static_assert(kT3Ring >= kT3Lag + 2, "mbarrier ring shorter than the drift the waits allow");

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                   (unsigned)__cvta_generic_to_shared(b))
               : "memory");
}
// true once the phase with the given parity has completed (acquire at CTA scope)
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, "
      "p;\n\t}"
      : "=r"(r)
      : "r"((unsigned)__cvta_generic_to_shared(b)), "r"(parity)
      : "memory");
  return r != 0;
}
// Monotone progress publication: flag = max(flag, v) with release semantics at GPU scope.
__device__ __forceinline__ void atom_max_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.max.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
template <int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void trail3_body(const Params& P, typename Prec::S* __restrict__ f, int* status,
                                            long long* t_dev, const FusedArgs& A, unsigned long long t) {
  constexpr int Q = 19;
  using R = typename Prec::R;
  using S_ = typename Prec::S;
  using PsiT = typename Prec::PsiT;
  using L = Lat<Q>;
  __shared__ unsigned long long mbar[kT3Ring];
  __shared__ int nbr[kF3MaxNbr];
  __shared__ int n_nbr;

  const int tid = threadIdx.x, b = blockIdx.x;
  const int r0 = A.range[b], S = A.range[b + 1] - r0;
  const int nx = P.nx, nz = P.nz;
  // progress value: planes collided + 1, at most nz + 1 in a launch
  const unsigned long long base = t * (unsigned long long)(nz + 2);
  const PsiT* __restrict__ psi_cur = (const PsiT*)A.psi_ring + (size_t)(t & 1) * P.N;
  PsiT* psi_next = (PsiT*)A.psi_ring + (size_t)((t + 1) & 1) * P.N;
  if (tid == 0) {
    for (int i = 0; i < kT3Ring; ++i) mbar_init(&mbar[i], (unsigned)blockDim.x);
    int n = 0;
    while (n < kF3MaxNbr && A.nbr[b * kF3MaxNbr + n] >= 0) {
      nbr[n] = A.nbr[b * kF3MaxNbr + n];
      ++n;
    }
    n_nbr = n;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  int err = 0;
  bool ok = true;
  // the per-site work is out of line: the march's own state then does not stay live across the
  // collision's registers (the collision spills 8-24 bytes per site instead of several hundred)
  auto collide = [&](int z) {
#pragma unroll 1
    for (int i = tid; i < S; i += kT3Threads) {
      const int xy = r0 + i;
      collide_site<Q, NC, Prec, MRT, PAR, LBM_T3_CS>(P, f, psi_cur, xy % nx, xy / nx, z, nullptr);
    }
  };
  auto stage = [&](int z) {
#pragma unroll 1
    for (int i = tid; i < S; i += kT3Threads) {
      const int xy = r0 + i;
      Site st;
      st.set_xyz(P, xy % nx, xy / nx, z);
      PsiT v;
      err |= site_psi<Q, NC, Prec, 1 - PAR>(P, f, st, v);
      psi_next[st.idx] = v;
    }
  };
  // this CTA's collisions of plane z (and of every plane before it) are complete
  auto wait_cta = [&](int z) {
    unsigned it = 0;
    while (!mbar_test(&mbar[z % kT3Ring], (unsigned)((z / kT3Ring) & 1))) {
      if (++it > kSpinLimit) {
        ok = false;
        return;
      }
    }
  };
  // every neighbour CTA has collided plane z (lanes poll one neighbour each, the warp waits)
  auto wait_nbrs = [&](int z) {
    const int lane = tid & 31;
    bool mine = true;
    if (ok && lane < n_nbr) {
      const unsigned long long target = base + (unsigned long long)z + 1;
      const unsigned long long* fl = &A.flags[nbr[lane]];
      unsigned it = 0;
      while (ld_acquire_u64(fl) < target) {
        if (++it > kSpinLimit) {
          mine = false;
          break;
        }
        __nanosleep(64);
      }
    }
    __syncwarp();  // orders the warp's later loads after the polling lanes' acquires
    ok = __all_sync(0xffffffffu, mine) && ok;
  };
  // After its arrival on plane z's mbarrier each warp checks whether the phase is complete;
  // the warp whose arrival completed it (it sees the phase done, with every other thread's
  // writes acquired) publishes z at once, as a monotone maximum, so the CTA's visible progress
  // never lags its collisions.
  auto arrive_publish = [&](int z) {
    mbar_arrive(&mbar[z % kT3Ring]);
    if ((tid & 31) == 0 && mbar_test(&mbar[z % kT3Ring], (unsigned)((z / kT3Ring) & 1)) && b != A.silent_block)
      atom_max_release_u64(&A.flags[b], base + (unsigned long long)z + 1);
  };

  for (int k = 0; k < nz; ++k) {
    collide(k);
    arrive_publish(k);
    const int p = k - kT3Lag;
    if (p >= 1 && p <= nz - 2) {
      wait_cta(p + 1);
      wait_nbrs(p + 1);
      if (!__all_sync(0xffffffffu, ok)) ok = false;
      if (ok) stage(p);
    }
  }
  // the planes whose stage needs the end of the march: nz - LAG .. nz - 1, and plane 0 (it
  // reads slots that plane nz - 1's collision writes)
  wait_cta(nz - 1);
  wait_nbrs(nz - 1);
  ok = __all_sync(0xffffffffu, ok);
  if (ok) {
    for (int p = nz - kT3Lag < 1 ? 1 : nz - kT3Lag; p < nz; ++p) stage(p);
    stage(0);
  }
  if (!ok) err |= ST_TIMEOUT;
  // finish: the last CTA of the launch folds the pending status and advances the step
  if (err) atomicOr(A.pending, err);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const int pend = *(volatile int*)A.pending;
      // the collisions of step t are complete unless a wait timed out (state undefined then);
      // a psi error belongs to step t + 1, which becomes the failing step
      if (!(pend & ST_TIMEOUT)) *t_dev += 1;
      if (pend) *status |= pend;
      *A.pending = 0;
      *A.done = 0;
    }
  }
}

template <int NC, class Prec, int MRT>
__global__ void __maxnreg__(LBM_T3_MAXREG)
    k_trail3(const __grid_constant__ Params P, typename Prec::S* __restrict__ f, int* status, long long* t_dev,
             const __grid_constant__ FusedArgs A) {
  if (*(volatile int*)status) return;  // a previous step failed: do nothing
  const unsigned long long t = (unsigned long long)*(volatile long long*)t_dev;
  if (t & 1)
    trail3_body<NC, Prec, MRT, 1>(P, f, status, t_dev, A, t);
  else
    trail3_body<NC, Prec, MRT, 0>(P, f, status, t_dev, A, t);
}

}  // namespace lbm
