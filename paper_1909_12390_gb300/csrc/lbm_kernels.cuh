// Kernels of the two-kernel step (pseudo-potential pass, then force + collide + in-place
// stream) and of the context's set-up and read-back, templated on the lattice, the number of
// components and the storage precision. Included once per lattice by lbm_d2q9.cu and
// lbm_d3q19.cu, which instantiate the dispatch tables.
#pragma once

#include <cuda_runtime.h>

#include "lbm_core.cuh"
#include "lbm_ops.h"

namespace lbm {

struct PrecF64 {
  using S = double;  // stored population
  using R = double;  // arithmetic of moments, force and collision
  using PsiT = double;
};
struct PrecF32S {
  using S = float;
  using R = float;
  using PsiT = float;
};

constexpr int kBlock = 256;

__device__ __forceinline__ void raise_status(int* status, int bit) { atomicOr(status, bit); }

// ---------------------------------------------------------------------------------------
// Pass 1: cell-volume densities (S1), EOS (S2) and pseudo-potential (S3) of every site.
template <int Q, int NC, class Prec>
__global__ void __launch_bounds__(kBlock) k_psi(const Params P, const typename Prec::S* __restrict__ f,
                                                typename Prec::PsiT* __restrict__ psi, int* status,
                                                int parity) {
  using R = typename Prec::R;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  if (*(volatile int*)status) return;
  Site s;
  s.set(P, idx);
  R d[NC];
  For<0, NC>::run([&]<int C>() {
    R acc = 0;
    For<0, Q>::run([&]<int A>() { acc += (R)f[AA<Q>::template read_slot<A>(P, s, idx, parity, C)]; });
    d[C] = acc;
  });
  double rho[NC];
  R rho_t = 0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    rho[i] = P.rho_ref[i] + (double)d[i];
    rho_t += (R)P.rho_ref[i] + d[i];
  }
  EosOut<NC> e = eos_pr<NC>(P, rho);
  R psi2;
  if constexpr (sizeof(R) == 8) {
    psi2 = P.cpsi * (e.pD / e.Dd - rho_t * (1.0 / 3.0));
  } else {
    // the quotient and everything after it are well conditioned: FP32, like the stored psi
    psi2 = (float)P.cpsi * ((float)e.pD / (float)e.Dd - rho_t * (1.0f / 3.0f));
  }
  if (!isfinite(psi2) || !isfinite(rho_t)) {
    raise_status(status, ST_NONFINITE);
    return;
  }
  if (!(e.B < 1.0) || psi2 < (R)0) {
    raise_status(status, ST_PSI_DOMAIN);
    return;
  }
  psi[idx] = (typename Prec::PsiT)sqrt(psi2);
}

// ---------------------------------------------------------------------------------------
// Pass 2: total force (S4), split (S5), Guo-forced BGK or MRT collision and in-place AA
// streaming (S6).
template <int Q, int NC, class Prec, int MRT>
__global__ void __launch_bounds__(kBlock) k_collide(const Params P, typename Prec::S* __restrict__ f,
                                                    const typename Prec::PsiT* __restrict__ psi,
                                                    const int* status, long long* t_dev, int parity) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  constexpr int D = L::D;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  if (*(volatile const int*)status) return;
  // the step counter advances only for steps whose pseudo-potential pass succeeded
  if (idx == 0) *t_dev += 1;
  Site s;
  s.set(P, idx);

  R fl[NC][Q];
  For<0, NC>::run([&]<int C>() {
    For<0, Q>::run([&]<int A>() { fl[C][A] = (R)f[AA<Q>::template read_slot<A>(P, s, idx, parity, C)]; });
  });

  // S4: F = -beta G psi(x) sum_a w_a psi(x+e_a) e_a - (1-beta)/2 G sum_a w_a psi^2(x+e_a) e_a
  R s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
  For<1, Q>::run([&]<int A>() {
    R pn = (R)psi[s.nb(P, L::e(A, 0), L::e(A, 1), L::e(A, 2))];
    R wp = (R)L::w(A) * pn;
    R wq = wp * pn;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (L::e(A, d) > 0) { s1[d] += wp; s2[d] += wq; }
      if (L::e(A, d) < 0) { s1[d] -= wp; s2[d] -= wq; }
    }
  });
  const R p0 = (R)psi[idx];
  const R c1 = (R)(-P.beta * P.G), c2 = (R)(-0.5 * (1.0 - P.beta) * P.G);
  R F[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) F[d] = c1 * p0 * s1[d] + c2 * s2[d];

  // S1 moments: shifted densities delta_c = rho_c - rho_ref_c and total momentum j
  R dl[NC], j[3] = {0, 0, 0};
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    R acc = 0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      acc += fl[c][a];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        if (L::e(a, d) > 0) j[d] += fl[c][a];
        if (L::e(a, d) < 0) j[d] -= fl[c][a];
      }
    }
    dl[c] = acc;
  }
  R rc[NC], rho = 0, gs = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    rc[c] = (R)P.rho_ref[c] + dl[c];
    rho += rc[c];
    gs += (R)P.gamma[c] * rc[c];
  }
  // barycentric velocity with the Guo half force
  R u[3] = {0, 0, 0};
  const R irho = (R)1 / rho;
#pragma unroll
  for (int d = 0; d < D; ++d) u[d] = (j[d] + (R)0.5 * F[d]) * irho;
  R uu = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) uu += u[d] * u[d];

  // per-site equilibrium polynomial P_a = 3 e.u + 9/2 (e.u)^2 - 3/2 u.u and the Guo term of the
  // total force Fb_a = w_a [3 (e_a - u).F + 9 (e_a.u)(e_a.F)]; component s uses chi_s Fb_a.
  R Pa[Q], Fb[Q];
  R uF = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) uF += u[d] * F[d];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    R eu = 0, eF = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (L::e(a, d) > 0) { eu += u[d]; eF += F[d]; }
      if (L::e(a, d) < 0) { eu -= u[d]; eF -= F[d]; }
    }
    Pa[a] = eu * ((R)3 + (R)4.5 * eu) - (R)1.5 * uu;
    Fb[a] = (R)L::w(a) * ((R)3 * (eF - uF) + (R)9 * eu * eF);
  }

  const R om = (R)P.omega;
  const R gk = (R)1 - (R)0.5 * om;
  const R igs = (R)1 / gs;
  For<0, NC>::run([&]<int C>() {
    const R chi = (R)P.gamma[C] * rc[C] * igs;  // S5
    R g[Q], out[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      // non-equilibrium part: f - f_eq in the stored (shifted) variables
      g[a] = fl[C][a] - (R)L::w(a) * (dl[C] + rc[C] * Pa[a]);
      out[a] = fl[C][a] - om * g[a] + gk * chi * Fb[a];
    }
    if constexpr (MRT) {
      // rows with their own rate: f* -= sum_k M_ka lam_k (M q)_k, q = g + chi Fb / 2
      R q[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) q[a] = g[a] + (R)0.5 * chi * Fb[a];
#pragma unroll
      for (int i = 0; i < L::NK; ++i) {
        const int k = L::krow(i);
        R mq = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          if (L::m(k, a) != 0) mq += (R)L::m(k, a) * q[a];
        }
        mq *= (R)P.lam[i];
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          if (L::m(k, a) != 0) out[a] -= (R)L::m(k, a) * mq;
        }
      }
    }
    For<0, Q>::run([&]<int A>() {
      f[AA<Q>::template write_slot<A>(P, s, idx, parity, C)] = (typename Prec::S)out[A];
    });
  });
}

// ---------------------------------------------------------------------------------------
// Set-up and read-back kernels (FP64 arithmetic, not on the timed path).

// f = f_eq(rho_c, u) of Eq. equilibrium(a), stored in the even layout, shift subtracted.
template <int Q, int NC, class Prec>
__global__ void k_init(const Params P, typename Prec::S* f, const double* __restrict__ rho,
                       const double* __restrict__ u) {
  using L = Lat<Q>;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  double uv[3] = {0, 0, 0}, uu = 0;
  if (u) {
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
      uv[d] = u[d * P.N + idx];
      uu += uv[d] * uv[d];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double r = rho[c * P.N + idx];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      double eu = 0;
#pragma unroll
      for (int d = 0; d < L::D; ++d) eu += L::e(a, d) * uv[d];
      double feq = r * L::w(a) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
      f[((int64_t)c * Q + a) * P.N + idx] = (typename Prec::S)(feq - L::w(a) * P.rho_ref[c]);
    }
  }
}

// canonical FP64 populations <-> storage
template <int Q, int NC, class Prec>
__global__ void k_get_f(const Params P, const typename Prec::S* __restrict__ f, double* out, int parity) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  Site s;
  s.set(P, idx);
  For<0, NC>::run([&]<int C>() {
    For<0, Q>::run([&]<int A>() {
      out[((int64_t)C * Q + A) * P.N + idx] =
          (double)f[AA<Q>::template read_slot<A>(P, s, idx, parity, C)] + Lat<Q>::w(A) * P.rho_ref[C];
    });
  });
}

template <int Q, int NC, class Prec>
__global__ void k_set_f(const Params P, typename Prec::S* f, const double* __restrict__ in) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int64_t k = ((int64_t)c * Q + a) * P.N + idx;
      f[k] = (typename Prec::S)(in[k] - Lat<Q>::w(a) * P.rho_ref[c]);
    }
}

// Macroscopic fields of the current state; psi must hold this state's pseudo-potential.
template <int Q, int NC, class Prec>
__global__ void k_fields(const Params P, const typename Prec::S* __restrict__ f,
                         const typename Prec::PsiT* __restrict__ psi, double* rho_out, double* u_out,
                         double* p_out, double* psi_out, int parity) {
  using L = Lat<Q>;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  Site s;
  s.set(P, idx);
  double rc[NC], j[3] = {0, 0, 0}, rho = 0;
  For<0, NC>::run([&]<int C>() {
    double acc = 0;
    For<0, Q>::run([&]<int A>() {
      double v = (double)f[AA<Q>::template read_slot<A>(P, s, idx, parity, C)];
      acc += v;
#pragma unroll
      for (int d = 0; d < L::D; ++d) j[d] += L::e(A, d) * v;
    });
    rc[C] = P.rho_ref[C] + acc;
    rho += rc[C];
  });
  double s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
  For<1, Q>::run([&]<int A>() {
    double pn = (double)psi[s.nb(P, L::e(A, 0), L::e(A, 1), L::e(A, 2))];
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
      s1[d] += L::w(A) * pn * L::e(A, d);
      s2[d] += L::w(A) * pn * pn * L::e(A, d);
    }
  });
  const double p0 = (double)psi[idx];
  EosOut<NC> e = eos_pr<NC>(P, rc);
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (rho_out) rho_out[c * P.N + idx] = rc[c];
  for (int d = 0; d < 3; ++d) {
    double F = d < L::D ? -P.beta * P.G * p0 * s1[d] - 0.5 * (1.0 - P.beta) * P.G * s2[d] : 0.0;
    if (u_out) u_out[d * P.N + idx] = (j[d] + 0.5 * F) / rho;
  }
  if (p_out) p_out[idx] = e.pD / e.Dd;
  if (psi_out) psi_out[idx] = p0;
}

// Per-component mass: per-block partial sums in FP64, then one block sums the partials,
// both in a fixed order.
template <int Q, int NC, class Prec>
__global__ void __launch_bounds__(kBlock) k_mass_partial(const Params P, const typename Prec::S* __restrict__ f,
                                                         double* partial) {
  __shared__ double sh[kBlock];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int c = 0; c < NC; ++c) {
    double v = 0;
    if (idx < P.N) {
      // every slot of the component holds exactly one population (in either AA layout, and
      // opposite directions share a weight), so the slot-wise sum over the grid is the mass
      for (int a = 0; a < Q; ++a) v += (double)f[((int64_t)c * Q + a) * P.N + idx] + Lat<Q>::w(a) * P.rho_ref[c];
    }
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int st = kBlock / 2; st > 0; st >>= 1) {
      if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
      __syncthreads();
    }
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * NC + c] = sh[0];
    __syncthreads();
  }
}

__global__ void k_mass_final(const double* partial, int nblocks, int nc, double* out);

// ---------------------------------------------------------------------------------------
// Host launchers and the dispatch table of one (Q, NC, precision, collision).
template <int Q, int NC, class Prec, int MRT>
struct Launch {
  using S = typename Prec::S;
  using PsiT = typename Prec::PsiT;
  static unsigned blocks(const Params& P) { return (unsigned)((P.N + kBlock - 1) / kBlock); }
  static void psi(const Params& P, const void* f, void* ps, int* st, int parity, cudaStream_t s) {
    k_psi<Q, NC, Prec><<<blocks(P), kBlock, 0, s>>>(P, (const S*)f, (PsiT*)ps, st, parity);
  }
  static void collide(const Params& P, void* f, const void* ps, const int* st, long long* t_dev, int parity,
                      cudaStream_t s) {
    k_collide<Q, NC, Prec, MRT><<<blocks(P), kBlock, 0, s>>>(P, (S*)f, (const PsiT*)ps, st, t_dev, parity);
  }
  static void init(const Params& P, void* f, const double* rho, const double* u, cudaStream_t s) {
    k_init<Q, NC, Prec><<<blocks(P), kBlock, 0, s>>>(P, (S*)f, rho, u);
  }
  static void get_f(const Params& P, const void* f, double* out, int parity, cudaStream_t s) {
    k_get_f<Q, NC, Prec><<<blocks(P), kBlock, 0, s>>>(P, (const S*)f, out, parity);
  }
  static void set_f(const Params& P, void* f, const double* in, cudaStream_t s) {
    k_set_f<Q, NC, Prec><<<blocks(P), kBlock, 0, s>>>(P, (S*)f, in);
  }
  static void fields(const Params& P, const void* f, const void* ps, double* rho, double* u, double* p,
                     double* psi_out, int parity, cudaStream_t s) {
    k_fields<Q, NC, Prec><<<blocks(P), kBlock, 0, s>>>(P, (const S*)f, (const PsiT*)ps, rho, u, p, psi_out,
                                                       parity);
  }
  static void mass(const Params& P, const void* f, double* partial, double* out, cudaStream_t s) {
    unsigned nb = blocks(P);
    k_mass_partial<Q, NC, Prec><<<nb, kBlock, 0, s>>>(P, (const S*)f, partial);
    k_mass_final<<<1, kBlock, 0, s>>>(partial, (int)nb, NC, out);
  }
  static const Ops* table() {
    static const Ops ops = {psi, collide, init, get_f, set_f, fields, mass, (int)sizeof(S), (int)sizeof(PsiT)};
    return &ops;
  }
};

template <int Q, class Prec, int MRT>
const Ops* ops_nc(int nc) {
  switch (nc) {
    case 1: return Launch<Q, 1, Prec, MRT>::table();
    case 2: return Launch<Q, 2, Prec, MRT>::table();
    case 3: return Launch<Q, 3, Prec, MRT>::table();
    case 4: return Launch<Q, 4, Prec, MRT>::table();
  }
  return nullptr;
}

template <int Q>
const Ops* ops_for(int nc, int precision, int collision) {
  if (precision == 0) return collision ? ops_nc<Q, PrecF64, 1>(nc) : ops_nc<Q, PrecF64, 0>(nc);
  return collision ? ops_nc<Q, PrecF32S, 1>(nc) : ops_nc<Q, PrecF32S, 0>(nc);
}

}  // namespace lbm
