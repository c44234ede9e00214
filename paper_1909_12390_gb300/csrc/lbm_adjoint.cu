// Hand-written discrete adjoint of the BGK step (Eq. LBE with the Guo forcing of Eq.
// equilibrium, the split of Eq. distributionforce, the force of Eq. coupledMCforce and the EOS
// of Eq. MCPengRobinson), for gradients of a loss on the final cell-volume densities with
// respect to the binary interaction coefficients zeta_ij, the volatility coefficients gamma_i
// and the initial densities.
//
// Forward, per site x (t -> t + 1): rho_s = sum_a f_sa, j = sum e_a f_sa, psi(rho), F from the
// psi stencil, chi_s = gamma_s rho_s / Gam, u = (j + F/2)/rho,
//   f*_sa = (1 - w) f_sa + w feq_sa(rho_s, u) + gk chi_s Fb_a(u, F),  f_sa(x + e_a) = f*_sa(x).
// Reverse, given lam(t+1) = dL/df(t+1) (canonical layout):
//   lam*_sa(x) = lam_sa(x + e_a)                                          (un-stream)
//   with L0_s = sum_a w_a lam*_sa, L1_s = sum_a w_a lam*_sa e_a, L2_s = sum_a w_a lam*_sa e_a e_a:
//   ubar   = sum_s w rho_s (3 L1 + 9 L2 u - 3 u L0) + gk chi_s (-3 F L0 + 9 L2 F)
//   Fbar   = gk sum_s chi_s (3 L1 - 3 u L0 + 9 L2 u) + ubar / (2 rho)
//   chibar = gk (3 L1.F - 3 (u.F) L0 + 9 u.L2.F)
//   rbar_s = w (L0 + 3 L1.u + 9/2 u.L2.u - 3/2 u.u L0) - ubar.u / rho
//            + gamma_s (chibar_s - sum_k chibar_k chi_k) / Gam            (pass A)
//   psibar(y) = c1 Fbar(y).S1(y) + sum_a w_a e_a.Fbar(y - e_a) [c1 psi(y - e_a) + 2 c2 psi(y)]
//   rbB_s = (psibar / 2 psi) cpsi (dp/dn_s / M_s - 1/3)                    (pass B)
//   lam_sa(t) = (1 - w) lam*_sa + rbar_s + (ubar / rho).e_a + rbB_s
// lam is held as X_sa = (1 - w) lam*_sa + rbar_s + (ubar / rho).e_a, written by pass A from
// what it has at hand, and rbB_s, written by pass B, which is added wherever lam is read (the
// next pass A's gather, the final dL/drho(0)). So pass B reads neither the populations nor
// lam: only psi, Fbar and the densities pass A leaves behind.
// MRT (f* = f - K (f - feq) + (I - K/2) chi_s Fb with K = w I + M^T Lam M over the rows whose
// rate differs from w, M the orthogonal moment basis, so K is symmetric): the same formulas with
// the moments of mu = K lam* where BGK has w times those of lam*, and the moments of
// nu = lam* - mu / 2 where it has gk times them; X_sa = lam*_sa - mu_sa + rbar_s + (ubar/rho).e_a.
// Parameter gradients: dL/dgamma_k = sum_x rho_k (chibar_k - sum chibar chi) / Gam and
// dL/dzeta_ij = sum_x pbar n_i n_j sqrt(a_i alpha_i a_j alpha_j) / (1 + 2B - B^2), reduced in
// FP64 per block and summed on the host in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm.h"
#include "lbm_host.h"
#include "lbm_kernels.cuh"

namespace lbm {

constexpr int kAdjBlock = 256;  // 64 and 128 measured the same on the 256^2 adjoint workload

// Adds the block-wide sums of v[0..M) to out[0..M) in a fixed order: warp shuffles, then the
// warps' sums in warp order (red holds M * kAdjBlock / 32 doubles). Every thread of the block
// calls it; the last one at the end of a kernel.
template <int M>
__device__ __forceinline__ void block_add(double (&v)[M], double* red, double* out) {
  constexpr int W = kAdjBlock / 32;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    double x = v[m];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[m * W + (threadIdx.x >> 5)] = x;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double x = 0;
    for (int w = 0; w < W; ++w) x += red[threadIdx.x * W + w];
    out[threadIdx.x] += x;
  }
}

// Per-thread sums of M gradient terms of type R and their block-wide reduction into FP64 rows.
// FP64: plain FP64 sums and block_add. FP32: each sum is a pair of FP32 values (hi + lo,
// Knuth's TwoSum, about 48 bits) reduced over the warp by shuffles in the same pair
// arithmetic, the block's warp pairs then summed in FP64 by thread m, in warp order. GB300's
// FP64 pipe retires under two lanes per clock per SM, so a warp-shuffle tree of FP64 additions
// costs hundreds of cycles per value and warp; the pair arithmetic runs on the FP32 pipe.
template <class R, int M>
struct GradSum;
template <int M>
struct GradSum<double, M> {
  double v[M];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int m = 0; m < M; ++m) v[m] = 0;
  }
  __device__ __forceinline__ void add(int m, double t) { v[m] += t; }
  // red: M * kAdjBlock / 32 doubles of shared memory
  __device__ __forceinline__ void flush(double* red, double* out) { block_add<M>(v, red, out); }
};
// (hi, lo) + t with |lo| <= ulp(hi) / 2 kept: TwoSum of hi and t, the error folded into lo and
// renormalised (round to nearest, no contraction: additions only, each explicitly rounded)
__device__ __forceinline__ void ff_add(float& hi, float& lo, float thi, float tlo) {
  const float s = __fadd_rn(hi, thi);
  const float bb = __fadd_rn(s, -hi);
  float e = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bb)), __fadd_rn(thi, -bb));
  e = __fadd_rn(e, __fadd_rn(lo, tlo));
  hi = __fadd_rn(s, e);
  lo = __fadd_rn(e, -__fadd_rn(hi, -s));
}
template <int M>
struct GradSum<float, M> {
  float hi[M], lo[M];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int m = 0; m < M; ++m) hi[m] = lo[m] = 0.f;
  }
  __device__ __forceinline__ void add(int m, float t) { ff_add(hi[m], lo[m], t, 0.f); }
  __device__ __forceinline__ void flush(double* red, double* out) {
    constexpr int W = kAdjBlock / 32;
    float* rf = reinterpret_cast<float*>(red);  // 2 * M * W floats: the same bytes as M * W doubles
#pragma unroll
    for (int m = 0; m < M; ++m) {
      float h = hi[m], l = lo[m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, h, o), ol = __shfl_down_sync(0xffffffffu, l, o);
        ff_add(h, l, oh, ol);
      }
      if ((threadIdx.x & 31) == 0) {
        rf[(m * W + (threadIdx.x >> 5)) * 2] = h;
        rf[(m * W + (threadIdx.x >> 5)) * 2 + 1] = l;
      }
    }
    __syncthreads();
    if (threadIdx.x < M) {
      double x = 0;
      for (int w = 0; w < W; ++w)
        x += (double)rf[(threadIdx.x * W + w) * 2] + (double)rf[(threadIdx.x * W + w) * 2 + 1];
      out[threadIdx.x] += x;
    }
  }
};

template <int Q, int NC, class Prec, int PAR>
__device__ __forceinline__ void load_site(const Params& P, const typename Prec::S* __restrict__ f, const Site& s,
                                          typename Prec::R (&rc)[NC], typename Prec::R (&j)[3]) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  j[0] = j[1] = j[2] = 0;
  For<0, NC>::run([&]<int C>() {
    const typename Prec::S* fc = comp_base<Q>(f, P, C);
    R acc = 0;
    For<0, Q>::run([&]<int A>() {
      const R v = (R)fc[AA<Q>::template rd<A, PAR>(P, s)];
      acc += v;
#pragma unroll
      for (int d = 0; d < L::D; ++d) {
        if (L::e(A, d) > 0) j[d] += v;
        if (L::e(A, d) < 0) j[d] -= v;
      }
    });
    rc[C] = PC<R>::rho_ref(P, C) + acc;
  });
}

// Pass A at one site x (Site s, linear index idx), from lam*_sa(x) = lam_sa(x + e_a) given by
// lam_star(c, a): writes X of lam(t), Fbar (D) and the cell-volume densities (NC) at x and sets
// gt to the site's dL/dgamma terms.
// mu = K v for one component's Q values: K = w I + sum over the free rows k of M_k^T lam_k M_k
// (the forward collision's relaxation, symmetric for the orthogonal basis).
template <int Q, class R>
__device__ __forceinline__ void mrt_k_apply(const Params& P, const R (&v)[Q], R (&mu)[Q]) {
  using L = Lat<Q>;
  R mk[L::NK];
  For<0, L::NK>::run([&]<int I>() {
    constexpr int k = L::krow(I);
    R m = 0;
    For<0, Q>::run([&]<int A>() {
      constexpr int cm = L::m(k, A);
      if constexpr (cm != 0) m += (R)cm * v[A];
    });
    mk[I] = PC<R>::lam(P, I) * m;
  });
  const R om = PC<R>::omega(P);
  For<0, Q>::run([&]<int A>() {
    R x = om * v[A];
    For<0, L::NK>::run([&]<int I>() {
      constexpr int cm = L::m(L::krow(I), A);
      if constexpr (cm != 0) x += (R)cm * mk[I];
    });
    mu[A] = x;
  });
}

// Lattice moments m0 = sum_a w_a v_a, m1 = sum_a w_a v_a e_a, m2 = sum_a w_a v_a e_a e_a.
template <int Q, class R>
__device__ __forceinline__ void w_moments(const R (&v)[Q], R& m0, R (&m1)[3], R (&m2)[3][3]) {
  using L = Lat<Q>;
  m0 = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    m1[d] = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) m2[d][e] = 0;
  }
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const R lw = (R)L::w(a) * v[a];
    m0 += lw;
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
      m1[d] += lw * (R)L::e(a, d);
#pragma unroll
      for (int e = 0; e < L::D; ++e) m2[d][e] += lw * (R)(L::e(a, d) * L::e(a, e));
    }
  }
}

template <int Q, int NC, class Prec, int PAR, int MRT, class LamStar>
__device__ __forceinline__ void adj_a_site(const Params& P, const typename Prec::S* __restrict__ f,
                                           const typename Prec::PsiT* __restrict__ psi, const Site& s, int64_t idx,
                                           const LamStar& lam_star, typename Prec::R* __restrict__ X_out,
                                           typename Prec::R* Fbar, typename Prec::R* rho_out, typename Prec::R (&gt)[NC]) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  constexpr int D = L::D;
  R rc[NC], j[3];
  load_site<Q, NC, Prec, PAR>(P, f, s, rc, j);
  // forward force
  R s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
#pragma unroll
  for (int a = 1; a < Q; ++a) {
    const R pn = (R)psi[s.nb(P, L::e(a, 0), L::e(a, 1), L::e(a, 2))];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      s1[d] += (R)L::w(a) * pn * (R)L::e(a, d);
      s2[d] += (R)L::w(a) * pn * pn * (R)L::e(a, d);
    }
  }
  const R p0 = (R)psi[idx];
  R F[3] = {0, 0, 0}, u[3] = {0, 0, 0};
  R rho = 0, gs = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    rho += rc[c];
    gs += PC<R>::gamma(P, c) * rc[c];
  }
  const R irho = (R)1 / rho, igs = (R)1 / gs;  // the divisions of this pass, once
#pragma unroll
  for (int d = 0; d < D; ++d) {
    F[d] = PC<R>::c1(P) * p0 * s1[d] + PC<R>::c2(P) * s2[d];
    u[d] = (j[d] + (R)0.5 * F[d]) * irho;
  }
  R uu = 0, uF = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    uu += u[d] * u[d];
    uF += u[d] * F[d];
  }
  const R om = PC<R>::omega(P), gk = PC<R>::gk(P);
  R ub[3] = {0, 0, 0}, Fd[3] = {0, 0, 0}, chib[NC], rb[NC], chi[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    chi[c] = PC<R>::gamma(P, c) * rc[c] * igs;
    if constexpr (MRT) {
      // the feq terms contract with mu = K lam*, the Guo terms with nu = lam* - mu / 2
      R ls[Q], mu[Q], nu[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) ls[a] = lam_star(c, a);
      mrt_k_apply<Q, R>(P, ls, mu);
#pragma unroll
      for (int a = 0; a < Q; ++a) nu[a] = ls[a] - (R)0.5 * mu[a];
      R M0, M1[3], M2[3][3], N0, N1[3], N2[3][3];
      w_moments<Q, R>(mu, M0, M1, M2);
      w_moments<Q, R>(nu, N0, N1, N2);
      R M2u[3] = {0, 0, 0}, N2u[3] = {0, 0, 0}, N2F[3] = {0, 0, 0};
#pragma unroll
      for (int d = 0; d < D; ++d)
#pragma unroll
        for (int e2 = 0; e2 < D; ++e2) {
          M2u[d] += M2[d][e2] * u[e2];
          N2u[d] += N2[d][e2] * u[e2];
          N2F[d] += N2[d][e2] * F[e2];
        }
      R M1u = 0, uM2u = 0, N1F = 0, uN2F = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        M1u += M1[d] * u[d];
        uM2u += u[d] * M2u[d];
        N1F += N1[d] * F[d];
        uN2F += u[d] * N2F[d];
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        ub[d] += rc[c] * ((R)3 * M1[d] + (R)9 * M2u[d] - (R)3 * u[d] * M0) +
                 chi[c] * ((R)-3 * F[d] * N0 + (R)9 * N2F[d]);
        Fd[d] += chi[c] * ((R)3 * N1[d] - (R)3 * u[d] * N0 + (R)9 * N2u[d]);
      }
      chib[c] = (R)3 * N1F - (R)3 * uF * N0 + (R)9 * uN2F;
      rb[c] = M0 + (R)3 * M1u + (R)4.5 * uM2u - (R)1.5 * uu * M0;
      continue;
    }
    R L0 = 0, L1[3] = {0, 0, 0}, L2[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const R lw = (R)L::w(a) * lam_star(c, a);
      L0 += lw;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        L1[d] += lw * (R)L::e(a, d);
#pragma unroll
        for (int e2 = 0; e2 < D; ++e2) L2[d][e2] += lw * (R)(L::e(a, d) * L::e(a, e2));
      }
    }
    R L2u[3] = {0, 0, 0}, L2F[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int e2 = 0; e2 < D; ++e2) {
        L2u[d] += L2[d][e2] * u[e2];
        L2F[d] += L2[d][e2] * F[e2];
      }
    R L1u = 0, L1F = 0, uL2u = 0, uL2F = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      L1u += L1[d] * u[d];
      L1F += L1[d] * F[d];
      uL2u += u[d] * L2u[d];
      uL2F += u[d] * L2F[d];
    }
#pragma unroll
    for (int d = 0; d < D; ++d) {
      ub[d] += om * rc[c] * ((R)3 * L1[d] + (R)9 * L2u[d] - (R)3 * u[d] * L0) +
               gk * chi[c] * ((R)-3 * F[d] * L0 + (R)9 * L2F[d]);
      Fd[d] += gk * chi[c] * ((R)3 * L1[d] - (R)3 * u[d] * L0 + (R)9 * L2u[d]);
    }
    chib[c] = gk * ((R)3 * L1F - (R)3 * uF * L0 + (R)9 * uL2F);
    rb[c] = om * (L0 + (R)3 * L1u + (R)4.5 * uL2u - (R)1.5 * uu * L0);
  }
  R ubu = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) ubu += ub[d] * u[d];
  R cc = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) cc += chib[c] * chi[c];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    rb[c] += -ubu * irho + PC<R>::gamma(P, c) * (chib[c] - cc) * igs;
    gt[c] = rc[c] * (chib[c] - cc) * igs;
    rho_out[c * P.N + idx] = rc[c];
  }
  R jb[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    Fbar[d * P.N + idx] = Fd[d] + (R)0.5 * ub[d] * irho;
    jb[d] = ub[d] * irho;
  }
  // X of lam(t); lam* is gathered again (L1)
  if constexpr (MRT) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      R ls[Q], mu[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) ls[a] = lam_star(c, a);
      mrt_k_apply<Q, R>(P, ls, mu);
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        R v = ls[a] - mu[a] + rb[c];
#pragma unroll
        for (int d = 0; d < D; ++d) v += jb[d] * (R)L::e(a, d);
        X_out[((int64_t)c * Q + a) * P.N + idx] = v;
      }
    }
    return;
  }
  const R w1 = (R)1 - om;
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      R v = w1 * lam_star(c, a) + rb[c];
#pragma unroll
      for (int d = 0; d < D; ++d) v += jb[d] * (R)L::e(a, d);
      X_out[((int64_t)c * Q + a) * P.N + idx] = v;
    }
}

// Pass A: collision adjoint at every site x, from lam(t + 1) = X + rbB. Writes X of lam(t),
// Fbar (D) and the cell-volume densities (NC) per site, and the per-block partial sums of
// dL/dgamma.
template <int Q, int NC, class Prec, int PAR, int MRT>
__global__ void __launch_bounds__(kAdjBlock) k_adj_a(const Params P, const typename Prec::S* __restrict__ f,
                                                     const typename Prec::PsiT* __restrict__ psi,
                                                     const typename Prec::R* __restrict__ X,
                                                     const typename Prec::R* __restrict__ rbB,
                                                     typename Prec::R* __restrict__ X_out, typename Prec::R* Fbar,
                                                     typename Prec::R* rho_out, double* gpart) {
  using L = Lat<Q>;
  __shared__ double red[NC * kAdjBlock / 32];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  GradSum<typename Prec::R, NC> gg;
  gg.zero();
  if (idx < P.N) {
    Site s;
    s.set(P, (uint32_t)idx);
    // lam*_sa(x) = lam_sa(x + e_a) = X_sa(x + e_a) + rbB_s(x + e_a)
    auto lam_star = [&](int c, int a) {
      const int64_t y = s.nb(P, L::e(a, 0), L::e(a, 1), L::e(a, 2));
      return X[((int64_t)c * Q + a) * P.N + y] + rbB[(int64_t)c * P.N + y];
    };
    typename Prec::R gt[NC];
    adj_a_site<Q, NC, Prec, PAR, MRT>(P, f, psi, s, idx, lam_star, X_out, Fbar, rho_out, gt);
#pragma unroll
    for (int c = 0; c < NC; ++c) gg.add(c, gt[c]);
  }
  // per-block partial sums of dL/dgamma, fixed order
  gg.flush(red, gpart + (int64_t)blockIdx.x * NC);
}

// Pass B at one site y (Site s, linear index idx): rbB of lam(t) (NC) into rb, and the site's
// dL/dzeta_ij terms (NC x NC) into kt.
template <int Q, int NC, class Prec>
__device__ __forceinline__ void adj_b_site(const Params& P, const typename Prec::PsiT* __restrict__ psi,
                                           const typename Prec::R* __restrict__ Fbar,
                                           const typename Prec::R* __restrict__ rho, const Site& s, int64_t idx,
                                           typename Prec::R (&rb)[NC], typename Prec::R (&kt)[NC * NC]) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  constexpr int D = L::D;
  R rc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) rc[c] = rho[c * P.N + idx];
  const R p0 = (R)psi[idx];
  // psibar(y) = c1 Fbar(y).S1(y) + sum_a w_a e_a.Fbar(y - e_a) [c1 psi(y - e_a) + 2 c2 psi(y)]
  R pb = 0;
  R S1[3] = {0, 0, 0};
#pragma unroll
  for (int a = 1; a < Q; ++a) {
    const int64_t yp = s.nb(P, L::e(a, 0), L::e(a, 1), L::e(a, 2));
    const int64_t ym = s.nb(P, -L::e(a, 0), -L::e(a, 1), -L::e(a, 2));
    const R pp = (R)psi[yp], pm = (R)psi[ym];
    R eFm = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      S1[d] += (R)L::w(a) * pp * (R)L::e(a, d);
      eFm += (R)L::e(a, d) * Fbar[d * P.N + ym];
    }
    pb += (R)L::w(a) * eFm * (PC<R>::c1(P) * pm + (R)2 * PC<R>::c2(P) * p0);
  }
#pragma unroll
  for (int d = 0; d < D; ++d) pb += PC<R>::c1(P) * Fbar[d * P.N + idx] * S1[d];
  // psi = sqrt(psi2), psi2 = cpsi (p - rho / 3): the EOS derivative, in the arithmetic of
  // the state (FP32 for FP32-shifted storage: its inputs carry FP32 precision and its terms
  // cancel at most a few-fold, so it keeps about 7 digits, far inside what the gradient
  // needs; GB300's FP64 pipe would make it the bottleneck of the reverse step). The zeta
  // gradient is accumulated in FP64.
  const R psi2b = pb / ((R)2 * p0);
  const R pbar = PC<R>::cpsi(P) * psi2b;
  auto cst = [&](const double& d, const float& f) -> R {
    if constexpr (sizeof(R) == 4)
      return f;
    else
      return d;
  };
  R n[NC], nt = 0, B = 0, A2 = 0, An[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    n[i] = rc[i] * PC<R>::invM(P, i);
    nt += n[i];
    B += cst(P.b[i], P.b_f[i]) * n[i];
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    An[i] = 0;
#pragma unroll
    for (int k = 0; k < NC; ++k) An[i] += cst(P.Qa[i * 4 + k], P.Qa_f[i * 4 + k]) * n[k];
    A2 += n[i] * An[i];
  }
  const R d1 = (R)1 - B, d2 = (R)1 + (R)2 * B - B * B;
  // dp/dn_i = RT/d1 + n RT b_i/d1^2 - 2 An_i/d2 + A2 (2 - 2B) b_i/d2^2, one division
  const R RT = cst(P.RT, P.RT_f);
  const R r12 = (R)1 / (d1 * d2);
  const R id1 = d2 * r12, id2 = d1 * r12;
  const R e0 = RT * id1;
  const R eb = nt * RT * id1 * id1 + A2 * ((R)2 - (R)2 * B) * id2 * id2;
  const R ea = (R)2 * id2;
  const R t3 = pbar * (R)(1.0 / 3.0);
  const R q = pbar * id2;
  R ns[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) ns[i] = n[i] * cst(P.sa[i], P.sa_f[i]);
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const R dpdn = e0 + eb * cst(P.b[i], P.b_f[i]) - ea * An[i];
    rb[i] = pbar * dpdn * PC<R>::invM(P, i) - t3;
#pragma unroll
    for (int k = 0; k < NC; ++k) kt[i * NC + k] = q * ns[i] * ns[k];
  }
}

// Pass B: force / pseudo-potential / EOS adjoint, rbB of lam(t) per site and component.
// kpart receives the per-block partial sums of dL/dzeta_ij (NC x NC).
template <int Q, int NC, class Prec>
__global__ void __launch_bounds__(kAdjBlock) k_adj_b(const Params P, const typename Prec::PsiT* __restrict__ psi,
                                                     const typename Prec::R* __restrict__ Fbar,
                                                     const typename Prec::R* __restrict__ rho,
                                                     typename Prec::R* __restrict__ rbB, double* kpart) {
  using R = typename Prec::R;
  __shared__ double red[NC * NC * kAdjBlock / 32];
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  GradSum<R, NC * NC> kg;
  kg.zero();
  if (idx < P.N) {
    Site s;
    s.set(P, (uint32_t)idx);
    R rb[NC], kt[NC * NC];
    adj_b_site<Q, NC, Prec>(P, psi, Fbar, rho, s, idx, rb, kt);
#pragma unroll
    for (int i = 0; i < NC; ++i) rbB[i * P.N + idx] = rb[i];
#pragma unroll
    for (int k = 0; k < NC * NC; ++k) kg.add(k, kt[k]);
  }
  kg.flush(red, kpart + (int64_t)blockIdx.x * NC * NC);
}

// Pass B of lam(t + 1) fused with pass A of the step t -> t + 1, D2Q9: one tile of
// kAbTX x kAbTY sites per block. The block first computes rbB(t + 1) on the tile and the ring
// of sites around it into shared memory (the ring's values are computed by the neighbouring
// tiles as well; only the tile's own sites add to the dL/dzeta sums), then pass A at the
// tile's sites with lam*(x) = X(t + 1)(x + e_a) + rbB(t + 1)(x + e_a), rbB from shared memory.
// The per-site arithmetic is that of the separate passes (the same device functions). Pass B
// reads Fbar and the densities of t + 1 (F_in, rho_in) while pass A writes those of t (F_out,
// rho_out), so they are separate buffers.
#ifndef LBM_ADJ_FUSED
#define LBM_ADJ_FUSED 1  // 0: D2Q9 runs the two passes as separate launches too
#endif
constexpr int kAbTX = 32, kAbTY = 8;
static_assert(kAbTX * kAbTY == kAdjBlock, "block_add sums over kAdjBlock threads");

template <int NC, class Prec, int PAR, int MRT>
__global__ void __launch_bounds__(kAdjBlock)
    k_adj_ab(const Params P, const typename Prec::S* __restrict__ f, const typename Prec::PsiT* __restrict__ psi_t,
             const typename Prec::PsiT* __restrict__ psi_t1, const typename Prec::R* __restrict__ X,
             typename Prec::R* __restrict__ X_out, const typename Prec::R* __restrict__ F_in,
             typename Prec::R* __restrict__ F_out, const typename Prec::R* __restrict__ rho_in,
             typename Prec::R* __restrict__ rho_out, double* gpart, double* kpart) {
  using R = typename Prec::R;
  using L = Lat<9>;
  constexpr int HX = kAbTX + 2, HY = kAbTY + 2, NH = HX * HY;
  __shared__ R rbs[NC][NH];
  __shared__ double red_g[NC * kAdjBlock / 32];
  __shared__ double red_k[NC * NC * kAdjBlock / 32];
  const int tid = threadIdx.x;
  const int tiles_x = (P.nx + kAbTX - 1) / kAbTX;
  const int x0 = (int)(blockIdx.x % tiles_x) * kAbTX, y0 = (int)(blockIdx.x / tiles_x) * kAbTY;
  GradSum<R, NC * NC> kg;
  kg.zero();
  for (int h = tid; h < NH; h += kAdjBlock) {
    const int hx = h % HX, hy = h / HX;
    const int gx = ((x0 - 1 + hx) % P.nx + P.nx) % P.nx, gy = ((y0 - 1 + hy) % P.ny + P.ny) % P.ny;
    const int64_t idx = (int64_t)gy * P.nx + gx;
    Site s;
    s.set(P, (uint32_t)idx);
    R rb[NC], kt[NC * NC];
    adj_b_site<9, NC, Prec>(P, psi_t1, F_in, rho_in, s, idx, rb, kt);
#pragma unroll
    for (int c = 0; c < NC; ++c) rbs[c][h] = rb[c];
    const bool own = hx >= 1 && hx <= kAbTX && hy >= 1 && hy <= kAbTY && x0 + hx - 1 < P.nx && y0 + hy - 1 < P.ny;
    if (own) {
#pragma unroll
      for (int k = 0; k < NC * NC; ++k) kg.add(k, kt[k]);
    }
  }
  __syncthreads();
  GradSum<R, NC> gg;
  gg.zero();
  const int lx = tid % kAbTX, ly = tid / kAbTX;
  const int x = x0 + lx, y = y0 + ly;
  if (x < P.nx && y < P.ny) {
    const int64_t idx = (int64_t)y * P.nx + x;
    Site s;
    s.set(P, (uint32_t)idx);
    auto lam_star = [&](int c, int a) {
      const int64_t yn = s.nb(P, L::e(a, 0), L::e(a, 1), 0);
      return X[((int64_t)c * 9 + a) * P.N + yn] + rbs[c][(ly + 1 + L::e(a, 1)) * HX + lx + 1 + L::e(a, 0)];
    };
    R gt[NC];
    adj_a_site<9, NC, Prec, PAR, MRT>(P, f, psi_t, s, idx, lam_star, X_out, F_out, rho_out, gt);
#pragma unroll
    for (int c = 0; c < NC; ++c) gg.add(c, gt[c]);
  }
  gg.flush(red_g, gpart + (int64_t)blockIdx.x * NC);
  kg.flush(red_k, kpart + (int64_t)blockIdx.x * NC * NC);
}

// lam(T)_sa(x) = dL/drho_s(x) for every a (X = dL/drho, rbB = 0);
// dL/drho(0)_s(x) = sum_a w_a lam(0)_sa(x), lam = X + rbB.
template <int Q, int NC, class Prec>
__global__ void k_adj_seed(const Params P, const double* __restrict__ drho, typename Prec::R* X,
                           typename Prec::R* rbB) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  for (int c = 0; c < NC; ++c) {
    for (int a = 0; a < Q; ++a) X[((int64_t)c * Q + a) * P.N + idx] = (typename Prec::R)drho[c * P.N + idx];
    rbB[c * P.N + idx] = 0;
  }
}

template <int Q, int NC, class Prec>
__global__ void k_adj_init_grad(const Params P, const typename Prec::R* __restrict__ X,
                                const typename Prec::R* __restrict__ rbB, double* drho0) {
  using R = typename Prec::R;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  for (int c = 0; c < NC; ++c) {
    double acc = 0;
    const R r = rbB[c * P.N + idx];
    for (int a = 0; a < Q; ++a) acc += Lat<Q>::w(a) * (double)(R)(X[((int64_t)c * Q + a) * P.N + idx] + r);
    drho0[c * P.N + idx] = acc;
  }
}

struct AdjFns {  // same layout as the declaration in lbm_capi.cu
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

template <int Q, int NC, class Prec, int MRT>
struct AdjLaunch {
  using R = typename Prec::R;
  using S = typename Prec::S;
  using PsiT = typename Prec::PsiT;
  static unsigned blocks(const Params& P) { return (unsigned)((P.N + kAdjBlock - 1) / kAdjBlock); }
  static void seed(const Params& P, const double* d, void* X, void* rbB, cudaStream_t s) {
    k_adj_seed<Q, NC, Prec><<<blocks(P), kAdjBlock, 0, s>>>(P, d, (R*)X, (R*)rbB);
  }
  static void pass_a(const Params& P, const void* f, const void* psi, const void* X, const void* rbB, void* Xo,
                     void* Fb, void* rho, int parity, double* gp, cudaStream_t s) {
    auto k = parity ? k_adj_a<Q, NC, Prec, 1, MRT> : k_adj_a<Q, NC, Prec, 0, MRT>;
    k<<<blocks(P), kAdjBlock, 0, s>>>(P, (const S*)f, (const PsiT*)psi, (const R*)X, (const R*)rbB, (R*)Xo, (R*)Fb,
                                      (R*)rho, gp);
  }
  static void pass_b(const Params& P, const void* psi, const void* Fb, const void* rho, void* rbB, double* kp,
                     cudaStream_t s) {
    k_adj_b<Q, NC, Prec><<<blocks(P), kAdjBlock, 0, s>>>(P, (const PsiT*)psi, (const R*)Fb, (const R*)rho, (R*)rbB,
                                                         kp);
  }
  static unsigned tiles(const Params& P) {
    return (unsigned)(((P.nx + kAbTX - 1) / kAbTX) * ((P.ny + kAbTY - 1) / kAbTY));
  }
  static void pass_ab(const Params& P, const void* f, const void* psi_t, const void* psi_t1, const void* X, void* Xo,
                      const void* Fi, void* Fo, const void* ri, void* ro, void* rbB, int parity, double* gp,
                      double* kp, cudaStream_t s) {
    if constexpr (Q == 9 && LBM_ADJ_FUSED) {
      auto k = parity ? k_adj_ab<NC, Prec, 1, MRT> : k_adj_ab<NC, Prec, 0, MRT>;
      k<<<tiles(P), kAdjBlock, 0, s>>>(P, (const S*)f, (const PsiT*)psi_t, (const PsiT*)psi_t1, (const R*)X, (R*)Xo,
                                       (const R*)Fi, (R*)Fo, (const R*)ri, (R*)ro, gp, kp);
    } else {
      pass_b(P, psi_t1, Fi, ri, rbB, kp, s);
      pass_a(P, f, psi_t, X, rbB, Xo, Fo, ro, parity, gp, s);
    }
  }
  static void init_grad(const Params& P, const void* X, const void* rbB, double* d, cudaStream_t s) {
    k_adj_init_grad<Q, NC, Prec><<<blocks(P), kAdjBlock, 0, s>>>(P, (const R*)X, (const R*)rbB, d);
  }
  static unsigned rows(const Params& P) { return Q == 9 ? std::max(blocks(P), tiles(P)) : blocks(P); }
  static const AdjFns* table() {
    static const AdjFns t = {seed, pass_a, pass_b, pass_ab, init_grad, rows, (int)sizeof(R)};
    return &t;
  }
};

template <int Q, class Prec, int MRT>
const AdjFns* adj_nc(int nc) {
  switch (nc) {
    case 1: return AdjLaunch<Q, 1, Prec, MRT>::table();
    case 2: return AdjLaunch<Q, 2, Prec, MRT>::table();
    case 3: return AdjLaunch<Q, 3, Prec, MRT>::table();
    case 4: return AdjLaunch<Q, 4, Prec, MRT>::table();
  }
  return nullptr;
}

template <int MRT>
const AdjFns* adj_coll(int Q, int nc, int precision) {
  if (Q == 9) return precision == LBM_FP64 ? adj_nc<9, PrecF64, MRT>(nc) : adj_nc<9, PrecF32S, MRT>(nc);
  return precision == LBM_FP64 ? adj_nc<19, PrecF64, MRT>(nc) : adj_nc<19, PrecF32S, MRT>(nc);
}

const AdjFns* adj_fns(int Q, int nc, int precision, int mrt) {
  return mrt ? adj_coll<1>(Q, nc, precision) : adj_coll<0>(Q, nc, precision);
}

}  // namespace lbm
