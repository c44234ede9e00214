// Fused D3Q19 step over plane ranges (k_fused3): one persistent cooperative launch per step.
//
// Worker w (two per CTA) owns the contiguous range [range[w], range[w+1]) of the flattened
// (y, x) index of a z plane and marches z = 0 .. nz-1, with psi computed LEAD planes ahead of the collision
// (LEAD = LBM_F3_LEAD). Before the march it computes psi of plane nz - 1 and of planes
// 0 .. LEAD - 1. Iteration k then
//   1. reads the populations of plane k + LEAD of its range from DRAM (the psi stage): the
//      densities of every site and from them the mixture EOS and psi, written to the psi
//      plane buffer;
//   2. publishes its progress (psi done up to plane k + LEAD) with st.release.gpu and waits
//      (bounded ld.acquire.gpu polls) until every worker owning a neighbour site has psi of
//      plane k + 1; with LEAD = 2 the neighbours published that an iteration earlier, so they
//      may lag by one iteration without stalling this worker;
//   3. collides and streams plane k in place: psi of the 18 neighbours from the plane buffers
//      (through L2), the populations re-read from L2 (LEAD iterations after the psi stage
//      read them; one iteration of the whole grid reads ~15 MB at 256^2 sites per plane).
// psi planes 1 .. nz-2 live in a ring of kF3Ring planes; plane 0 and plane nz-1 have their own
// buffers because plane nz-1's collision needs plane 0's psi from before the step and plane 0's
// collision needs plane nz-1's. A site's psi depends only on the populations it reads, and in
// the AA pattern every site reads and writes its own set of slots, so psi of any site may be
// computed at any time before that site's collision.
//
// Safety of the ring: a worker writing plane k + LEAD in iteration k has seen (its wait of
// iteration k - 1) every neighbour's psi of plane k, so each neighbour has passed the psi stage
// of iteration k - LEAD and collides plane k - LEAD or later, reading planes k - LEAD - 1 and
// up; with kF3Ring >= 2 LEAD + 2 the slot of plane k + LEAD is none of the planes
// k - LEAD - 1 .. k + LEAD - 1. Deadlock freedom: every wait targets progress that each
// neighbour publishes before its own wait of the same or an earlier iteration, and the
// cooperative launch makes all workers co-resident; every wait is bounded anyway (kSpinLimit
// polls), after which the step reports a timeout.
#pragma once

namespace lbm {

constexpr int kF3WorkersPerCta = 2;  // workers (plane ranges) per CTA
constexpr int kF3FlagSets = 1;       // progress counters per worker

// planes of look-ahead between a worker's psi stage and its collision: at 256^3 (D3Q19 MRT,
// three FP32-shifted components) 1, 2, 3 measured 3.45, 3.19-3.25 and 3.38 ms per step
#ifndef LBM_F3_LEAD
#define LBM_F3_LEAD 2
#endif
// One CTA per SM of two workers, each of 7 warps (kF3Worker threads) with its own plane range,
// named barriers and progress flag. Worker 1 starts after worker 0's first psi stage, so that
// in steady state one worker's psi stage (DRAM reads and the FP64 EOS) overlaps the other's
// collision (FP32 arithmetic and L2 traffic). An SM sub-partition's 16 K registers hold four
// warps of 128 registers or three of 168: workers of 224 threads (LBM_F3_WORKER) run at 128
// registers, workers of 192 at 168.
#ifndef LBM_F3_WORKER
#define LBM_F3_WORKER 224
#endif
constexpr int kF3Worker = LBM_F3_WORKER;
constexpr int kF3Threads = 2 * kF3Worker;
constexpr int kF3Bound = kF3Threads <= 384 ? 384 : 512;  // launch bound: 168 or 128 registers
static_assert(kF3Worker % 32 == 0 && kF3Threads <= 512, "worker size");
constexpr int kF3Lead = LBM_F3_LEAD;  // planes between the psi stage and the collision
constexpr int kF3Ring = 8;            // psi planes in the ring
constexpr int kF3MaxNbr = 16;         // neighbour workers of one worker
static_assert(kF3Lead >= 1 && kF3Ring >= 2 * kF3Lead + 2, "psi ring too short for the look-ahead");

// Named barrier of one worker (ids 1 and 2; 0 is __syncthreads) and its AND-reduction form.
__device__ __forceinline__ void f3_bar(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kF3Worker) : "memory");
}
__device__ __forceinline__ bool f3_bar_and(int id, bool v) {
  unsigned r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.and.pred p, %2, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((unsigned)v), "r"(id), "r"(kF3Worker)
      : "memory");
  return r != 0;
}

template <int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void fused3_body(const Params& P, typename Prec::S* __restrict__ f, int* status,
                                            long long* t_dev, const FusedArgs& A, unsigned long long t) {
  constexpr int Q = 19;
  using R = typename Prec::R;
  using PsiT = typename Prec::PsiT;
  using L = Lat<Q>;
  __shared__ int nbr_s[2][kF3MaxNbr];
  __shared__ int n_nbr_s[2];

  const int half = threadIdx.x >= kF3Worker ? 1 : 0;
  const int tid = threadIdx.x - half * kF3Worker;
  const int w = 2 * blockIdx.x + half;  // worker
  const int bar = 1 + half;
  const int r0 = A.range[w], S = A.range[w + 1] - r0;
  int* nbr = nbr_s[half];
  const int nx = P.nx, nz = P.nz, nxy = P.nx * P.ny;
  // progress value: last plane with psi published + 2, at most nz + LEAD + 1 in a launch
  const unsigned long long base = t * (unsigned long long)(nz + kF3Lead + 2);
  PsiT* ring = (PsiT*)A.psi_ring;
  auto plane = [&](int z) -> PsiT* {
    z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    if (z == 0) return ring + (size_t)kF3Ring * nxy;
    if (z == nz - 1) return ring + (size_t)(kF3Ring + 1) * nxy;
    return ring + (size_t)(z % kF3Ring) * nxy;
  };
  if (tid < kF3MaxNbr) nbr[tid] = A.nbr[w * kF3MaxNbr + tid];
  f3_bar(bar);
  if (tid == 0) {
    int n = 0;
    while (n < kF3MaxNbr && nbr[n] >= 0) ++n;
    n_nbr_s[half] = n;
  }

  int err = 0;
  bool ok = true;
  // psi stage of plane z (psi written when put; the plane's populations come through L2 for
  // the collision, which recomputes the site moments: that pass brings all of a site's
  // populations into L1 with every load in flight before the per-component passes)
  auto stage = [&](int z, bool put) {
    PsiT* dst = plane(z);
    for (int i = tid; i < S; i += kF3Worker) {
      const int xy = r0 + i;
      Site st;
      st.set_xyz(P, xy % nx, xy / nx, z);
      R dl[NC];
      site_densities<Q, NC, Prec, PAR>(P, f, st, dl);
      if (put) {
        PsiT v;
        err |= site_psi_dl<NC, Prec>(P, dl, v);
        dst[xy] = v;
      }
    }
  };
  auto publish = [&](int s_) {
    f3_bar(bar);
    if (tid == 0 && w != A.silent_block) st_release_u64(&A.flags[w], base + (unsigned long long)s_);
  };
  auto wait = [&](int s_) {
    bool mine = true;
    if (ok && tid < n_nbr_s[half]) {
      const unsigned long long target = base + (unsigned long long)s_;
      const unsigned long long* fl = &A.flags[nbr[tid]];
      unsigned it = 0;
      while (ld_acquire_u64(fl) < target) {
        if (++it > kSpinLimit) {
          mine = false;
          break;
        }
        __nanosleep(64);
      }
    }
    ok = f3_bar_and(bar, mine && ok);
  };
  auto collide = [&](int z) {
    const PsiT* pl[3] = {plane(z - 1), plane(z), plane(z + 1)};
#pragma unroll 1
    for (int i = tid; i < S; i += kF3Worker) {
      const int xy = r0 + i;
      const int x = xy % nx, y = xy / nx;
      Site st;
      st.set_xyz(P, x, y, z);
      const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
      const int ym = (y == 0 ? P.ny - 1 : y - 1) * nx, yp = (y == P.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
      R pn[Q];
      For<0, Q>::run([&]<int A_>() {
        constexpr int ex = L::e(A_, 0), ey = L::e(A_, 1), ez = L::e(A_, 2);
        const int col = ex < 0 ? xm : (ex > 0 ? xp : x);
        const int row = ey < 0 ? ym : (ey > 0 ? yp : y0);
        pn[A_] = (R)__ldcg(pl[ez + 1] + row + col);
      });
      site_collide<Q, NC, Prec, MRT, PAR>(P, f, st, pn);
    }
  };

  // worker 1 starts once worker 0 has done its first psi stage (barrier 3 spans the CTA)
  if (half == 1) asm volatile("bar.sync 3, %0;" ::"r"(kF3Threads) : "memory");
  stage(nz - 1, true);
  if (half == 0) asm volatile("bar.arrive 3, %0;" ::"r"(kF3Threads) : "memory");
  for (int p = 0; p < kF3Lead && p < nz; ++p) stage(p, p < nz - 1);
  publish(kF3Lead + 1);
  for (int k = 0; k < nz; ++k) {
    const int q = k + kF3Lead;
    if (q < nz) stage(q, q < nz - 1);
    publish(q + 2);
    wait(k + 3);
    if (!ok) break;
    collide(k);
  }
  if (!ok) err |= ST_TIMEOUT;
  // finish: the last CTA of the launch folds the pending status and advances the step
  if (err) atomicOr(A.pending, err);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      const int pend = *(volatile int*)A.pending;
      if (pend)
        *status |= pend;
      else
        *t_dev += 1;
      *A.pending = 0;
      *A.done = 0;
    }
  }
}



// One CTA per SM; the launch bound sets the register budget (see kF3Bound).
template <int NC, class Prec, int MRT>
__global__ void __launch_bounds__(kF3Bound, 1)
    k_fused3(const Params P, typename Prec::S* __restrict__ f, int* status, long long* t_dev, const FusedArgs A) {
  if (*(volatile int*)status) return;  // a previous step failed: do nothing
  const unsigned long long t = (unsigned long long)*(volatile long long*)t_dev;
  if (t & 1)
    fused3_body<NC, Prec, MRT, 1>(P, f, status, t_dev, A, t);
  else
    fused3_body<NC, Prec, MRT, 0>(P, f, status, t_dev, A, t);
}

}  // namespace lbm
