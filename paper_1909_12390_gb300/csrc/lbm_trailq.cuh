// Task-queue one-pass D3Q19 step (k_trailq): one launch per step whose CTAs take the step's
// tasks from a ticket counter, the pseudo-potential of the NEXT step trailing the collisions.
//
// Each z plane is cut into nch chunks of A.smax consecutive sites of the flattened (y, x) index.
// Tasks are (1) the collision of chunk c of plane z (psi(t) of the 18 neighbours read from the
// current field, read-only in this launch) and (2) psi(t + 1) of chunk c of plane z into the
// other field. The densities of the state at t + 1 at a site are sums over slots written by the
// collisions of the sites around it (AA pattern), so task (2) of (z, c) needs the collisions of
// planes z - 1 .. z + 1 of chunk c and of the chunks holding its sites' in-plane neighbours.
// The host lists the tasks in a fixed ticket order: every collision in plane order, with the
// psi task of (z, c) placed after the collision of (z + 1 + lag, c), so every task a psi task
// needs has a smaller ticket; the psi tasks of planes whose neighbours wrap (0 and nz - 1) go
// last. A CTA takes the next ticket when it finishes a task (fetched one task ahead), so CTAs
// stay independent as the blocks of the two-kernel step's collide pass do, while psi(t + 1)
// re-reads populations written a few planes earlier, from L2.
//
// A collision task publishes its completion (per (plane, chunk) flag = t + 1, release at GPU
// scope after the CTA's barrier); a psi task polls the flags it needs (bounded acquire polls),
// then reads the populations through L2 only (ld.global.cg: another SM may have written them
// since this SM's L1 cached an earlier read of the same lines). Waits go only to smaller
// tickets, which are held by running CTAs: the CTA holding the smallest ticket that waits
// waits for tasks that are either collisions (which never wait) or not yet started by a CTA
// whose current task has a still smaller ticket, hence does not wait; so the queue cannot
// deadlock, and it needs no co-residency guarantee (CTAs that start after the tickets ran out
// exit at once). Every wait is bounded anyway (kSpinLimit polls), after which the step reports
// a timeout and later psi tasks skip their work.
//
// The result of a step is the same, bit for bit, as that of the two-kernel step: the collision
// is the same per-site code, and psi(t + 1) of a site is site_psi over the same slots. Errors of
// the psi(t + 1) tasks (EOS domain, non-finite) are folded into the status word by the last CTA:
// step t completed, and the next step is the failing one.
#pragma once

namespace lbm {

#ifndef LBM_TQ_THREADS
#define LBM_TQ_THREADS 128
#endif
constexpr int kTQThreads = LBM_TQ_THREADS;
// CTAs per SM (the collision's register budget: 65536 / (4 x 128) = 128 registers)
#ifndef LBM_TQ_BLOCKS
#define LBM_TQ_BLOCKS 4
#endif
// planes between a collision and the psi task placed after it in the ticket order. About 600
// tasks run at once (4 CTAs per SM), which spans nearly 5 planes of 512-site chunks at 256^2;
// a psi task placed closer than that waits for collisions still running. Measured at 256^3:
// lag 1 / 3 / 6: 3.45 / 2.49 / 2.40 ms per step (chunks of 512); chunks of 256 / 1024 / 2048 at
// lag 6: 2.49 / 2.49 / 3.01 ms
#ifndef LBM_TQ_LAG
#define LBM_TQ_LAG 6
#endif
constexpr int kTQLag = LBM_TQ_LAG;
static_assert(kTQLag >= 1, "a psi task needs the collisions of the plane above it");
// sites per chunk (the unit of a task)
#ifndef LBM_TQ_CHUNK
#define LBM_TQ_CHUNK 512
#endif
constexpr int kTQChunk = LBM_TQ_CHUNK;
// population stores of the collision tasks: 1 evict-first, 2 write-back (kept in L2 for the
// psi tasks)
#ifndef LBM_TQ_CS
#define LBM_TQ_CS 2
#endif

__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(const volatile int*)p; }

// The two kinds of task: the collisions of one chunk, psi of the next step over one chunk.
// Inlined: out of line (each its own function, 28-40 B of spills against 450 B) the step
// measured 2.51 ms against 2.40 ms at 256^3.
template <int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void tq_collide_chunk(const Params& P, typename Prec::S* __restrict__ f,
                                                 const typename Prec::PsiT* __restrict__ psi_cur, int z, int lo,
                                                 int hi) {
  const int nx = P.nx;
#pragma unroll 1
  for (int i = lo + (int)threadIdx.x; i < hi; i += kTQThreads) {
    const int y = i / nx;
    collide_site<19, NC, Prec, MRT, PAR, LBM_TQ_CS>(P, f, psi_cur, i - y * nx, y, z, nullptr);
  }
}
template <int NC, class Prec, int PAR>
__device__ __forceinline__ int tq_psi_chunk(const Params& P, const typename Prec::S* __restrict__ f,
                                            typename Prec::PsiT* __restrict__ psi_next, int z, int lo, int hi) {
  const int nx = P.nx;
  int err = 0;
#pragma unroll 1
  for (int i = lo + (int)threadIdx.x; i < hi; i += kTQThreads) {
    const int y = i / nx;
    Site st;
    st.set_xyz(P, i - y * nx, y, z);
    typename Prec::PsiT v;
    err |= site_psi<19, NC, Prec, PAR, 1>(P, f, st, v);
    psi_next[st.idx] = v;
  }
  return err;
}

template <int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void trailq_body(const Params& P, typename Prec::S* __restrict__ f, int* status,
                                            long long* t_dev, const FusedArgs& A, unsigned long long t) {
  using PsiT = typename Prec::PsiT;
  __shared__ int s_tk[2];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int nx = P.nx, nz = P.nz, nch = A.nch, TS = A.smax, T = A.ntask;
  const int nxy = nx * P.ny;
  const unsigned long long epoch = t + 1;
  const PsiT* __restrict__ psi_cur = (const PsiT*)A.psi_ring + (size_t)(t & 1) * P.N;
  PsiT* psi_next = (PsiT*)A.psi_ring + (size_t)((t + 1) & 1) * P.N;

  int err = 0;
  if (tid == 0) s_tk[0] = (int)atomicAdd(A.ticket, 1u);
  __syncthreads();
  int buf = 0;
  int k = s_tk[0];
  while (k < T) {
    // the next ticket, fetched while this task runs (read after the closing barrier)
    if (tid == 0) s_tk[buf ^ 1] = (int)atomicAdd(A.ticket, 1u);
    const int task = __ldg(A.tasks + k);
    if (task >= 0) {
      const int z = task / nch, c = task - z * nch;
      tq_collide_chunk<NC, Prec, MRT, PAR>(P, f, psi_cur, z, c * TS, min(c * TS + TS, nxy));
      __syncthreads();  // the chunk's stores, ordered before thread 0's release below
      if (tid == 0 && c != A.silent_block) {
        __threadfence();
        st_release_u64(&A.flags[task], epoch);
      }
    } else {
      const int q = -task - 1, z = q / nch, c = q - z * nch;
      if (tid < 32) {
        const int* nb = A.nbr + (size_t)c * kF3MaxNbr;
        int nn = 0;
        while (nn < kF3MaxNbr && __ldg(nb + nn) >= 0) ++nn;
        const int per = 1 + nn;
        bool mine = !(ld_volatile_int(A.pending) & ST_TIMEOUT);
        for (int d = tid; mine && d < 3 * per; d += 32) {
          const int zz = (z + d / per - 1 + nz) % nz, j = d % per;
          const int cc = j == 0 ? c : __ldg(nb + j - 1);
          const unsigned long long* fl = &A.flags[(size_t)zz * nch + cc];
          unsigned it = 0;
          while (ld_acquire_u64(fl) < epoch) {
            if (++it > kSpinLimit || (ld_volatile_int(A.pending) & ST_TIMEOUT)) {
              mine = false;
              break;
            }
            __nanosleep(64);
          }
        }
        const bool all = __all_sync(0xffffffffu, mine);
        if (tid == 0) {
          s_ok = all;
          if (!all) atomicOr(A.pending, ST_TIMEOUT);
        }
      }
      __syncthreads();  // orders the block's loads below after the polling lanes' acquires
      if (s_ok) err |= tq_psi_chunk<NC, Prec, 1 - PAR>(P, f, psi_next, z, c * TS, min(c * TS + TS, nxy));
    }
    __syncthreads();  // s_tk[buf ^ 1] written; s_ok and s_tk[buf] free for reuse
    buf ^= 1;
    k = s_tk[buf];
  }
  // finish: the last CTA of the launch folds the pending status, advances the step and resets
  // the ticket counter (every other CTA has taken its last ticket by then)
  if (err) atomicOr(A.pending, err);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const int pend = ld_volatile_int(A.pending);
      // the collisions of step t are complete unless a wait timed out (psi(t + 1) undefined
      // then); a psi error belongs to step t + 1, which becomes the failing step
      if (!(pend & ST_TIMEOUT)) *t_dev += 1;
      if (pend) *status |= pend;
      *A.pending = 0;
      *A.done = 0;
      *A.ticket = 0;
    }
  }
}

template <int NC, class Prec, int MRT>
__global__ void __launch_bounds__(kTQThreads, LBM_TQ_BLOCKS)
    k_trailq(const __grid_constant__ Params P, typename Prec::S* __restrict__ f, int* status, long long* t_dev,
             const __grid_constant__ FusedArgs A) {
  if (*(volatile int*)status) return;  // a previous step failed: do nothing
  const unsigned long long t = (unsigned long long)*(volatile long long*)t_dev;
  if (t & 1)
    trailq_body<NC, Prec, MRT, 1>(P, f, status, t_dev, A, t);
  else
    trailq_body<NC, Prec, MRT, 0>(P, f, status, t_dev, A, t);
}

}  // namespace lbm
