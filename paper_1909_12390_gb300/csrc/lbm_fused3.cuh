// Fused D3Q19 step over plane ranges (k_fused3): one persistent cooperative launch per step.
//
// CTA b owns the contiguous range [range[b], range[b+1]) of the flattened (y, x) index of a
// z plane and marches z = 0 .. nz-1. Iteration k
//   1. reads the populations of plane k + 1 of its range once from DRAM (the psi stage): the
//      moments of every site (shifted densities and momentum, kept per thread for the
//      collision) and from them the mixture EOS and psi, written to the psi plane buffer;
//   2. publishes progress k + 2 (st.release.gpu) and waits (bounded ld.acquire.gpu polls) until
//      every CTA owning a neighbour site has published it too;
//   3. collides and streams plane k in place: psi of the 18 neighbours from the plane buffers
//      (through L2), the populations re-read from L2 (read one iteration before; one plane of
//      the whole grid is ~45 MB of traffic between the two reads).
// psi planes 1 .. nz-2 live in a ring of kF3Ring planes; plane 0 and plane nz-1 have their own
// buffers because plane nz-1's collision needs plane 0's psi from before the step and plane 0's
// collision needs plane nz-1's. A site's psi depends only on the populations it reads, and in
// the AA pattern every site reads and writes its own set of slots, so psi of any site may be
// computed at any time before that site's collision.
//
// Safety of the ring: a CTA writing plane k + 1 in iteration k has seen progress k + 1 from
// every neighbour, so each neighbour has finished the psi stage of iteration k - 1 and is at
// least colliding plane k - 1, which reads planes k - 2 .. k: with kF3Ring >= 4 the slot of
// plane k + 1 is none of them. Deadlock freedom: every CTA publishes stage s before it waits
// for stage s, and the cooperative launch makes all CTAs co-resident; every wait is bounded
// anyway (kSpinLimit polls), after which the step reports a timeout.
#pragma once

namespace lbm {

constexpr int kF3Threads = 224;  // 7 warps; two CTAs per SM at 144 registers
constexpr int kF3Ring = 8;       // psi planes in the ring
constexpr int kF3MaxNbr = 16;    // neighbour CTAs of one CTA

template <int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void fused3_body(const Params& P, typename Prec::S* __restrict__ f, int* status,
                                            long long* t_dev, const FusedArgs& A, unsigned long long t) {
  constexpr int Q = 19;
  using R = typename Prec::R;
  using PsiT = typename Prec::PsiT;
  using L = Lat<Q>;
  extern __shared__ __align__(16) unsigned char f3_smem[];
  R* mom = reinterpret_cast<R*>(f3_smem);  // [2][NC + 3][smax]: moments of the next two planes
  __shared__ int nbr[kF3MaxNbr];
  __shared__ int n_nbr;

  const int b = blockIdx.x;
  const int r0 = A.range[b], S = A.range[b + 1] - r0, SM = A.smax;
  const int nx = P.nx, nz = P.nz, nxy = P.nx * P.ny;
  const unsigned long long base = t * (unsigned long long)(nz + 1);
  PsiT* ring = (PsiT*)A.psi_ring;
  auto plane = [&](int z) -> PsiT* {
    z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    if (z == 0) return ring + (size_t)kF3Ring * nxy;
    if (z == nz - 1) return ring + (size_t)(kF3Ring + 1) * nxy;
    return ring + (size_t)(z % kF3Ring) * nxy;
  };
  if (threadIdx.x < kF3MaxNbr) nbr[threadIdx.x] = A.nbr[b * kF3MaxNbr + threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    while (n < kF3MaxNbr && nbr[n] >= 0) ++n;
    n_nbr = n;
  }

  int err = 0;
  bool ok = true;
  // psi stage of plane z: moments (kept in buffer buf when keep) and psi (written when put)
  auto stage = [&](int z, int buf, bool put, bool keep) {
    PsiT* dst = plane(z);
    R* m = mom + (size_t)buf * (NC + 3) * SM;
    for (int i = threadIdx.x; i < S; i += kF3Threads) {
      const int xy = r0 + i;
      Site st;
      st.set_xyz(P, xy % nx, xy / nx, z);
      R dl[NC], j[3];
      site_moments<Q, NC, Prec, PAR>(P, f, st, dl, j);
      if (put) {
        PsiT v;
        err |= site_psi_dl<NC, Prec>(P, dl, v);
        dst[xy] = v;
      }
      if (keep) {
#pragma unroll
        for (int c = 0; c < NC; ++c) m[c * SM + i] = dl[c];
#pragma unroll
        for (int d = 0; d < 3; ++d) m[(NC + d) * SM + i] = j[d];
      }
    }
  };
  auto publish = [&](int s_) {
    __syncthreads();
    if (threadIdx.x == 0 && b != A.silent_block) st_release_u64(&A.flags[b], base + (unsigned long long)s_);
  };
  auto wait = [&](int s_) {
    bool mine = true;
    if (ok && threadIdx.x < n_nbr) {
      const unsigned long long target = base + (unsigned long long)s_;
      const unsigned long long* fl = &A.flags[nbr[threadIdx.x]];
      unsigned it = 0;
      while (ld_acquire_u64(fl) < target) {
        if (++it > kSpinLimit) {
          mine = false;
          break;
        }
        __nanosleep(64);
      }
    }
    ok = __syncthreads_and(mine && ok) != 0;
  };
  auto collide = [&](int z, int buf) {
    const PsiT* pl[3] = {plane(z - 1), plane(z), plane(z + 1)};
    const R* m = mom + (size_t)buf * (NC + 3) * SM;
#pragma unroll 1
    for (int i = threadIdx.x; i < S; i += kF3Threads) {
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
      R dl[NC], j[3];
#pragma unroll
      for (int c = 0; c < NC; ++c) dl[c] = m[c * SM + i];
#pragma unroll
      for (int d = 0; d < 3; ++d) j[d] = m[(NC + d) * SM + i];
      site_collide_m<Q, NC, Prec, MRT, PAR>(P, f, st, pn, dl, j);
    }
  };

  // stage 1: psi of the last plane (plane 0's collision needs it) and of the first plane
  if (nz > 1) stage(nz - 1, 0, true, false);
  stage(0, 0, true, true);
  publish(1);
  for (int k = 0; k < nz; ++k) {
    if (k + 1 < nz) stage(k + 1, (k + 1) & 1, k + 1 < nz - 1, true);
    publish(k + 2);
    wait(k + 2);
    if (!ok) break;
    collide(k, k & 1);
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

// 144 registers: two CTAs of kF3Threads per SM (2 x 224 x 144 <= 65536)
template <int NC, class Prec, int MRT>
__global__ void __maxnreg__(144)
    k_fused3(const Params P, typename Prec::S* __restrict__ f, int* status, long long* t_dev, const FusedArgs A) {
  if (*(volatile int*)status) return;  // a previous step failed: do nothing
  const unsigned long long t = (unsigned long long)*(volatile long long*)t_dev;
  if (t & 1)
    fused3_body<NC, Prec, MRT, 1>(P, f, status, t_dev, A, t);
  else
    fused3_body<NC, Prec, MRT, 0>(P, f, status, t_dev, A, t);
}

}  // namespace lbm
