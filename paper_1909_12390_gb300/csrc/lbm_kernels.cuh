// Kernels of one time step, templated on the lattice, the number of components and the
// storage precision, and the context's set-up / read-back kernels. lbm_<lattice>_<storage>.cu
// instantiate the dispatch tables, one translation unit per lattice and storage type.
//
// Two step paths share the per-site bodies site_psi (S1-S3) and site_collide (S4-S6):
//   * two-kernel: k_psi over every site, then k_collide over every site;
//   * fused: k_fused, one persistent cooperative launch per step in which every block marches
//     its tile column along the slowest axis, computes psi once per site, publishes each plane
//     of psi with a release flag, waits (bounded) for its neighbour tiles' flags and then
//     collides and streams the plane in place.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

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
// Collide pass: threads per block and resident blocks per SM, which set its register budget
// (an SM sub-partition's 16 K registers: 4 warps of 128 or 3 of 168 registers).
#ifndef LBM_COLLIDE_THREADS
#define LBM_COLLIDE_THREADS 128
#endif
#ifndef LBM_COLLIDE_BLOCKS
#define LBM_COLLIDE_BLOCKS 4
#endif
// The D3Q19 FP64 collision is bound by GB300's FP64 pipe rather than by latency, so it trades
// resident warps for registers: at 2 blocks (up to 255 registers) it spills 56 B per thread
// instead of about 2 KB, and measured 37.21 ms per 256^3 collide pass against 37.50 ms at 4
// (3 blocks: 37.63 ms).
#ifndef LBM_COLLIDE_BLOCKS_F64
#define LBM_COLLIDE_BLOCKS_F64 2
#endif
constexpr int kCollideThreads = LBM_COLLIDE_THREADS;
constexpr int kCollideBlocks = LBM_COLLIDE_BLOCKS;
// threads per block of the staged collide pass (LBM_COLLIDE_STAGED), which is also the stride
// of its per-thread copies in shared memory
#ifndef LBM_COLLIDE_STAGED_THREADS
#define LBM_COLLIDE_STAGED_THREADS 64
#endif
constexpr int kStageThreads = LBM_COLLIDE_STAGED_THREADS;
template <int Q, class Prec>
constexpr int kCollideBlocksOf = Q == 19 && sizeof(typename Prec::R) == 8 ? LBM_COLLIDE_BLOCKS_F64 : kCollideBlocks;
// Per-pair values of a site shared by every component and both passes of the collision
// (w Pe, 3 w e.u, Fe, Fo): 1 computes them once per site and holds them in registers, 0
// recomputes them in each pass. At 256^3 (D3Q19 MRT, 3 components, FP32) option 1 measured
// 1.580 ms per collide pass against 1.626 ms; a per-thread shared-memory table measured 1.765 ms.
#ifndef LBM_COLLIDE_PAIRS
#define LBM_COLLIDE_PAIRS 1
#endif
// Pairs of opposite populations whose loads the collision's update pass issues together
// (all of them by default). At 256^3 (D3Q19 MRT, 3 components, FP32) k_collide measured
// 1.579 / 1.546 / 1.544 / 1.538 ms with groups of 1 / 3 / 5 / 9 pairs.
#ifndef LBM_COLLIDE_GROUP
#define LBM_COLLIDE_GROUP 9
#endif

// Programmatic dependent launch of the two-kernel step's passes: each is launched with the
// programmatic-serialization attribute, so that its blocks can be scheduled while the kernel
// before it in the stream is finishing. Every block first waits (griddepcontrol.wait) until that
// kernel has completed and its memory is visible, then lets the next pass be scheduled
// (griddepcontrol.launch_dependents). Nothing is read before the wait, so results do not
// change; only the launch gap between the passes is hidden. The attribute is given only when
// both passes of the step fit in one wave of resident blocks each: measured per step, the 256^2
// two-component droplet 8.14 -> 7.09 us and the 64^2 slab 13.5 -> 13.3 us, but the 512^2
// three-component droplet, whose collide pass takes several waves, 22.2 -> 23.1 us with the
// attribute on both passes and 22.3 -> 23.7 us with it on its single-wave psi pass alone.
// Without the attribute the wait returns at once. LBM_PDL = 0 launches every pass plainly.
#ifndef LBM_PDL
#define LBM_PDL 1
#endif
__device__ __forceinline__ void pdl_enter() {
#if LBM_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Population stores into global memory are marked evict-first (st.global.cs, GLOBAL = 1): the
// written populations are not read again in the step, and keeping them out of the way leaves L2
// to the populations still to be read. GLOBAL = 2 is a plain global store (st.global.wb), for a
// step that re-reads what it wrote from L2. GLOBAL = 0 selects a generic store, required when
// the populations live in shared memory (the batched kernel): st.global on a shared address is
// an address-space fault.
template <class Prec, int GLOBAL>
__device__ __forceinline__ void store_pop(typename Prec::S* p, typename Prec::R v) {
  if constexpr (GLOBAL == 1)
    __stcs(p, (typename Prec::S)v);
  else if constexpr (GLOBAL == 2)
    __stwb(p, (typename Prec::S)v);  // global memory, kept in L2 (write-back)
  else
    *p = (typename Prec::S)v;
}

// ---------------------------------------------------------------------------------------
// S2-S3 of one site from its shifted densities dl_c = rho_c - rho_ref_c: mixture
// Peng-Robinson EOS and pseudo-potential. Returns 0 or status bits; psi_out is 0 on error.
template <int NC, class Prec>
__device__ __forceinline__ int site_psi_dl(const Params& P, const typename Prec::R (&d)[NC],
                                           typename Prec::PsiT& psi_out) {
  using R = typename Prec::R;
  R rho_t = 0;
  R psi2;
  bool dom;  // B < 1
  if constexpr (sizeof(R) == 8) {
    double rho[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      rho[i] = P.rho_ref[i] + d[i];
      rho_t += rho[i];
    }
    EosOut<NC> e = eos_pr<NC>(P, rho);
    psi2 = P.cpsi * fmx(-rho_t, 1.0 / 3.0, e.pD / e.Dd);
    dom = e.B < 1.0;
  } else {
    float rc[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      rc[i] = P.rho_ref_f[i] + d[i];
      rho_t += rc[i];
    }
    EosOutF e = eos_pr_f32in<NC>(P, rc);
    // the quotient and everything after it are well conditioned: FP32, like the stored psi;
    // psi^2 = cpsi RT (p / RT - rho / (3 RT))
    const double pq[2] = {e.pD, e.Dd};
    float q[2];
    narrow_all<2>(pq, q);
    psi2 = P.cpsi_rt_f * fmx(-rho_t, P.c3rt_f, q[0] / q[1]);
    dom = e.ok;
  }
  psi_out = 0;
  if (!isfinite(psi2) || !isfinite(rho_t)) return ST_NONFINITE;
  if (!dom || psi2 < (R)0) return ST_PSI_DOMAIN;
  psi_out = (typename Prec::PsiT)sqrt(psi2);
  return 0;
}

// Shifted densities of one site, summed in the same order as site_moments (rest, then the
// pairs), so that every path computes bit-identical densities. CG = 1 loads through L2 only
// (ld.global.cg): for populations that other SMs wrote earlier in the same launch, which a
// line left in this SM's L1 by an earlier read could otherwise shadow.
template <int Q, int NC, class Prec, int PAR, int CG = 0>
__device__ __forceinline__ void site_densities(const Params& P, const typename Prec::S* __restrict__ f,
                                               const Site& s, typename Prec::R (&d)[NC]) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  For<0, NC>::run([&]<int C>() {
    const typename Prec::S* fc = comp_base<Q>(f, P, C);
    auto ld = [&](uint32_t o) -> R {
      if constexpr (CG)
        return (R)__ldcg(fc + o);
      else
        return (R)fc[o];
    };
    R acc = ld(AA<Q>::template rd<0, PAR>(P, s));
    For<0, L::NPAIR>::run([&]<int K>() {
      constexpr int a = L::pfirst(K), b = L::opp(a);
      acc += ld(AA<Q>::template rd<a, PAR>(P, s)) + ld(AA<Q>::template rd<b, PAR>(P, s));
    });
    d[C] = acc;
  });
}

// S1-S3 of one site: cell-volume densities, mixture Peng-Robinson EOS, pseudo-potential.
// Returns 0 or status bits; psi_out is 0 on error.
template <int Q, int NC, class Prec, int PAR, int CG = 0>
__device__ __forceinline__ int site_psi(const Params& P, const typename Prec::S* __restrict__ f, const Site& s,
                                        typename Prec::PsiT& psi_out) {
  typename Prec::R d[NC];
  site_densities<Q, NC, Prec, PAR, CG>(P, f, s, d);
  return site_psi_dl<NC, Prec>(P, d, psi_out);
}

// Hides a value from the optimiser (no instruction): what is computed from it afterwards is
// not merged with what was computed from it before.
__device__ __forceinline__ void opaque(float& x) { asm volatile("" : "+f"(x)); }
__device__ __forceinline__ void opaque(double& x) { asm volatile("" : "+d"(x)); }
__device__ __forceinline__ void opaque(Site& t) {
  asm volatile("" : "+r"(t.idx), "+r"(t.x), "+r"(t.y), "+r"(t.z));
  asm volatile("" : "+r"(t.xm), "+r"(t.xp), "+r"(t.ym), "+r"(t.yp), "+r"(t.zm), "+r"(t.zp));
}

// Population load that the optimiser keeps where it is written: a plain load of the same
// address (the moments pass read every population already) would be merged with the earlier
// one and keep Q * NC values in registers through the collision. The "memory" clobber keeps
// it ordered with the stores: in the in-place update of a pair (a, b) the new value for a
// goes to b's slot, and it must not be stored before b's value has been read. Generic addressing, so the
// same code serves populations in global and in shared memory.
__device__ __forceinline__ float ld_pop(const float* p) {
  float v;
  asm volatile("ld.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_pop(const double* p) {
  double v;
  asm volatile("ld.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}

// Split factors of Gong et al.'s comparison model (Eq. Gong) with the two pressures under the
// root put in the order that makes the difference non-negative, as the paper does to keep it
// real (Section 4.2): chi_i = c_i sqrt(|p0 - ph_i|) / sum_j c_j sqrt(|p0 - ph_j|), c_i the
// molar composition, ph_i the Peng-Robinson pressure of pure component i at the mixture's
// molar density n, p0 = n R T. FP64 (the pressures cancel).
template <int NC, class R>
__device__ __forceinline__ void gong_split(const Params& P, const R (&rc)[NC], R (&chi)[NC]) {
  double n[NC], nt = 0.0, w[NC], ws = 0.0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    n[i] = (double)rc[i] * P.invM[i];
    nt += n[i];
  }
  const double p0 = nt * P.RT;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    const double bn = P.b[i] * nt;
    const double ph = p0 / (1.0 - bn) - P.sa[i] * P.sa[i] * nt * nt / (1.0 + bn * (2.0 - bn));
    w[i] = n[i] / nt * sqrt(fabs(p0 - ph));
    ws += w[i];
  }
#pragma unroll
  for (int i = 0; i < NC; ++i) chi[i] = (R)(w[i] / ws);
}

// S1 moments of one site: shifted component densities dl_c = sum_a f_ca = rho_c - rho_ref_c
// and the total momentum j = sum_c sum_a e_a f_ca. The momentum is summed from the differences
// of opposite populations: near equilibrium the two are close, so in FP32 each difference is
// exact and j carries no rounding on the scale of the populations.
// SRC = 1: the site's populations were staged by its own thread in shared memory, component
// C's population a at stg[(C Q + a) kStageThreads] (k_collide_staged); 0: read from their slots.
template <int Q, int NC, class Prec, int PAR, int SRC = 0>
__device__ __forceinline__ void site_moments(const Params& P, const typename Prec::S* __restrict__ f, const Site& s,
                                             typename Prec::R (&dl)[NC], typename Prec::R (&j)[3],
                                             const float* stg = nullptr) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  j[0] = j[1] = j[2] = 0;
  For<0, NC>::run([&]<int C>() {
    const typename Prec::S* fc = comp_base<Q>(f, P, C);
    auto pop = [&]<int A>() -> R {
      if constexpr (SRC)
        return (R)stg[(C * Q + A) * kStageThreads];
      else
        return (R)fc[AA<Q>::template rd<A, PAR>(P, s)];
    };
    R acc = pop.template operator()<0>();
    For<0, L::NPAIR>::run([&]<int K>() {
      constexpr int a = L::pfirst(K), b = L::opp(a);
      const R va = pop.template operator()<a>();
      const R vb = pop.template operator()<b>();
      acc += va + vb;
      const R d = va - vb;
#pragma unroll
      for (int k = 0; k < L::D; ++k) {
        if (L::e(a, k) > 0) j[k] += d;
        if (L::e(a, k) < 0) j[k] -= d;
      }
    });
    dl[C] = acc;
  });
}

// The two members of a pair of opposite populations pass through identical arithmetic. In
// FP32 each such operation is one paired-FP32 instruction (fma / add / mul .f32x2 of
// Blackwell) rather than two; each lane rounds exactly like the scalar operation it replaces,
// so results do not change. FP64 (and LBM_COLLIDE_PACKED = 0) runs the two lanes as scalars.
#ifndef LBM_COLLIDE_PACKED
#define LBM_COLLIDE_PACKED 1
#endif
template <class R>
struct V2 {
  R x, y;
};
template <class R>
__device__ __forceinline__ V2<R> v2(R a, R b) {
  return {a, b};
}
__device__ __forceinline__ V2<float> fma2(V2<float> a, V2<float> b, V2<float> c) {
#if LBM_COLLIDE_PACKED
  const float2 r = __ffma2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y), make_float2(c.x, c.y));
  return {r.x, r.y};
#else
  return {fmx(a.x, b.x, c.x), fmx(a.y, b.y, c.y)};
#endif
}
__device__ __forceinline__ V2<float> add2(V2<float> a, V2<float> b) {
#if LBM_COLLIDE_PACKED
  const float2 r = __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  return {r.x, r.y};
#else
  return {a.x + b.x, a.y + b.y};
#endif
}
__device__ __forceinline__ V2<float> mul2(V2<float> a, V2<float> b) {
#if LBM_COLLIDE_PACKED
  const float2 r = __fmul2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
  return {r.x, r.y};
#else
  return {a.x * b.x, a.y * b.y};
#endif
}
__device__ __forceinline__ V2<double> fma2(V2<double> a, V2<double> b, V2<double> c) {
  return {fmx(a.x, b.x, c.x), fmx(a.y, b.y, c.y)};
}
__device__ __forceinline__ V2<double> add2(V2<double> a, V2<double> b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ V2<double> mul2(V2<double> a, V2<double> b) { return {a.x * b.x, a.y * b.y}; }

// Per-site values shared by every component's collision (S4, S5 and the velocity of
// Eq. equilibrium), computed once per site by site_prep and read by comp_collide.
template <int Q, int NC, class R, int PT>
struct SitePrep {
  R rc[NC], dl[NC], chis[NC];
  R u[3], F[3], uF, P0, F0;
  R pt_r[PT ? 4 * Lat<Q>::NPAIR : 1];
};

// e_a . v for a compile-time direction a (additions only).
template <int Q, int A, class R>
__device__ __forceinline__ R edot(const R (&v)[3]) {
  R x = 0;
#pragma unroll
  for (int d = 0; d < Lat<Q>::D; ++d) {
    if (Lat<Q>::e(A, d) > 0) x += v[d];
    if (Lat<Q>::e(A, d) < 0) x -= v[d];
  }
  return x;
}

template <int Q, int NC, class Prec, int PT = LBM_COLLIDE_PAIRS>
__device__ __forceinline__ void site_prep(const Params& P, const typename Prec::R (&pn)[Q],
                                          const typename Prec::R (&dl)[NC], const typename Prec::R (&j)[3],
                                          SitePrep<Q, NC, typename Prec::R, PT>& sp) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  constexpr int D = L::D;
  constexpr int NP = L::NPAIR;

  // S4: F = -beta G psi(x) sum_a w_a psi(x+e_a) e_a - (1-beta)/2 G sum_a w_a psi^2(x+e_a) e_a.
  // With psi_+ = psi(x + e_p), psi_- = psi(x - e_p) and sum_a w_a e_a = 0 it equals exactly
  //   F = -G [psi(x) S1 + (1-beta)/2 S2],  S1 = sum_p w_p e_p (psi_+ - psi_-),
  //                                        S2 = sum_p w_p e_p (psi_+ - psi_-)(psi_+ + psi_- - 2 psi(x)),
  // whose two terms do not cancel (S2 is a second-difference correction). In FP32 the textbook
  // form loses several ulps to that cancellation, and the rounding leaves a net force on the
  // periodic grid (zero in exact arithmetic) that accumulates into a drift of whole interfaces.
  // Weights are counted in 1/36.
  R S1[3] = {0, 0, 0}, S2[3] = {0, 0, 0};
  For<0, NP>::run([&]<int K>() {
    constexpr int a = L::pfirst(K), b = L::opp(a);
    constexpr int iw = L::c2(a) == 1 ? (Q == 9 ? 4 : 2) : 1;  // 36 w_a
    static_assert(iw / 36.0 - L::w(a) < 1e-15 && L::w(a) - iw / 36.0 < 1e-15);
    const R dp = pn[a] - pn[b];
    const R dc = dp * fmx((R)-2, pn[0], pn[a] + pn[b]);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      if (L::e(a, d) != 0) {
        S1[d] = fmx((R)(iw * L::e(a, d)), dp, S1[d]);
        S2[d] = fmx((R)(iw * L::e(a, d)), dc, S2[d]);
      }
    }
  });
  const R k1p = PC<R>::k1(P) * pn[0], k2 = PC<R>::k2(P);
  R* F = sp.F;
  F[0] = F[1] = F[2] = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) F[d] = fmx(k1p, S1[d], k2 * S2[d]);

  R (&rc)[NC] = sp.rc;
  R rho = 0, gs = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    rc[c] = PC<R>::rho_ref(P, c) + dl[c];
    rho += rc[c];
    gs = fmx(PC<R>::gamma(P, c), rc[c], gs);
  }
  // barycentric velocity with the Guo half force
  R* u = sp.u;
  u[0] = u[1] = u[2] = 0;
  const R irho = (R)1 / rho;
#pragma unroll
  for (int d = 0; d < D; ++d) u[d] = fmx((R)0.5, F[d], j[d]) * irho;
  R uu = 0, uF = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    uu = fmx(u[d], u[d], uu);
    uF = fmx(u[d], F[d], uF);
  }
  sp.uF = uF;
  // Per pair p the even / odd parts of P_a = 3 e.u + 9/2 (e.u)^2 - 3/2 u.u (Pe +- Po) and of
  // Fb_a = w_a [3 (e_a - u).F + 9 (e_a.u)(e_a.F)] (Fe +- Fo) are formed inside each
  // component's loop from e_p.u and e_p.F (a few adds; keeping them per site would hold
  // 2 (Q - 1) more registers through the component loop).
  const R P0 = -(R)1.5 * uu;
  const R F0 = -(R)(3.0 * L::w(0)) * uF;
  sp.P0 = P0;
  sp.F0 = F0;
  // per-pair values of the site (PT = 1): [0] Pe, [1] e.u, [2] Fe, [3] Fo
  auto pt = [&](int i, int k) -> R& { return sp.pt_r[PT ? i * NP + k : 0]; };
  if constexpr (PT) {
    For<0, NP>::run([&]<int K>() {
      constexpr int a = L::pfirst(K);
      const R eu = edot<Q, a>(sp.u);
      const R eF = edot<Q, a>(sp.F);
      pt(0, K) = fmx((R)4.5 * eu, eu, P0);
      pt(1, K) = eu;
      pt(2, K) = (R)L::w(a) * fmx((R)9 * eu, eF, (R)-3 * uF);
      pt(3, K) = (R)(3.0 * L::w(a)) * eF;
    });
  }
  // S5: split factors
  R (&chis)[NC] = sp.chis;
  if (P.split == 0) {
    const R igs = (R)1 / gs;
#pragma unroll
    for (int c = 0; c < NC; ++c) chis[c] = PC<R>::gamma(P, c) * rc[c] * igs;  // Eq. distributionforce
  } else {
    gong_split<NC, R>(P, rc, chis);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) sp.dl[c] = dl[c];
}

// S6 of component C at one site, given the site's shared values: Guo-forced BGK or MRT
// collision and the in-place AA write (see site_collide_m for the pair arrangement).
template <int Q, int NC, class Prec, int MRT, int PAR, int C, int GLOBAL = 1, int PT = LBM_COLLIDE_PAIRS,
          int SRC = 0>
__device__ __forceinline__ void comp_collide(const Params& P, typename Prec::S* __restrict__ f, const Site& s,
                                             const SitePrep<Q, NC, typename Prec::R, PT>& sp,
                                             typename Prec::S* fo = nullptr, const float* stg = nullptr) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  constexpr int NP = L::NPAIR;
  const R* rc = sp.rc;
  const R* dl = sp.dl;
  const R* u = sp.u;
  const R* F = sp.F;
  const R uF = sp.uF, P0 = sp.P0, F0 = sp.F0;
  auto pt = [&](int i, int k) -> R { return sp.pt_r[PT ? i * NP + k : 0]; };
  auto dot = [&](const R (&v)[3], auto a_) { return edot<Q, decltype(a_)::value>(v); };
  const R om = PC<R>::omega(P);
  const R gk = PC<R>::gk(P);
  const R chi = sp.chis[C];
  // Compiler-only barrier: the populations are re-read (from L1) rather than kept in
  // registers from the moments pass, which would cost Q * NC registers.
  asm volatile("" ::: "memory");
  const R gkchi = gk * chi;
  typename Prec::S* fc = comp_base<Q>(f, P, C);
  // the new values go to the same slots of fo when given (a step out of place: each site
  // writes exactly the slots it reads), else in place
  typename Prec::S* fcw = comp_base<Q>(fo ? fo : f, P, C);
  // Non-equilibrium part g = f - f_eq (stored variables) per pair: A is the even part of the
  // equilibrium (one value for both members), B the odd part; the BGK + Guo change is
  // d = gk chi Fb - omega g. For MRT a first pass accumulates the free-row moments of
  // q = g + chi Fb / 2 in pair form (q_a + q_b = g_a + g_b + chi Fe, q_a - q_b =
  // g_a - g_b + chi Fo; even rows through per-class sums, odd rows directly); the second
  // pass re-reads the populations (L1), forms d and the MRT correction and stores. Keeping
  // nothing per pair between the passes keeps the register count down.
  // Per-pair values are the same for every component and both passes. With PT = 1 they
  // come from the table computed once per site (4 registers per pair: about 9 instructions
  // per pair and pass fewer, and fewer spills at 128 registers). With PT = 0 u, F and u.F
  // pass through an empty asm, which makes them opaque per pass, so the values are
  // recomputed from them (a few FMAs per pair) instead of held.
  R uo[3], Fo_[3], uFo = uF, P0o = P0;
  // The site's addresses are likewise made opaque per pass. Besides bounding the registers,
  // this keeps the instruction stream of the collision the same in every kernel that
  // inlines it: without it the fused and two-kernel steps were measured to differ in the
  // last bit (the multiply-add contractions follow the instruction order).
  Site so = s;
  auto refresh = [&]() {
    so = s;
    opaque(so);
    if constexpr (!PT) {  // with the table, u, F and u.F are not needed after it is filled
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        uo[d] = u[d];
        Fo_[d] = F[d];
        opaque(uo[d]);
        opaque(Fo_[d]);
      }
      uFo = uF;
      P0o = P0;
      opaque(uFo);
      opaque(P0o);
    }
  };
  // 3 w_a rho_c per weight class (|e_a|^2 = 1, 2)
  const R b31 = (R)(3.0 * L::w(L::pfirst(0))) * rc[C], b32 = (R)(3.0 * L::w(L::pfirst(NP - 1))) * rc[C];
  static_assert(L::c2(L::pfirst(0)) == 1 && L::c2(L::pfirst(NP - 1)) == 2, "pair order");
  // g_a,b = v_a,b - w (dl + rho Pe) -+ 3 w rho e.u: each member in two multiply-adds, so the
  // large even part of the equilibrium is never rounded on its own. Rounding it first
  // (one ulp of the population, a biased error because w is inexact in binary) measured a
  // 6x larger error of the 20000-step FP32 droplet against the oracle.
  auto pair_g = [&](auto k_, R va, R vb, V2<R>& g, R& Fe, R& Fo) {
    constexpr int K = decltype(k_)::value;
    constexpr int a = L::pfirst(K);
    R Pe, eu;
    if constexpr (PT) {
      Pe = pt(0, K);
      eu = pt(1, K);
      Fe = pt(2, K);
      Fo = pt(3, K);
    } else {
      eu = dot(uo, std::integral_constant<int, a>{});
      const R eF = dot(Fo_, std::integral_constant<int, a>{});
      Pe = fmx((R)4.5 * eu, eu, P0o);
      Fe = (R)L::w(a) * fmx((R)9 * eu, eF, (R)-3 * uFo);
      Fo = (R)(3.0 * L::w(a)) * eF;
    }
    const R t = fmx(rc[C], Pe, dl[C]);
    const R b3 = L::c2(a) == 1 ? b31 : b32;
    const R mw = -(R)L::w(a);
    g = fma2(v2(-b3, b3), v2(eu, eu), fma2(v2(mw, mw), v2(t, t), v2(va, vb)));
  };
  // population A of this component: from its slot, or (SRC = 1) from the thread's staged copy
  auto ldp = [&]<int A>() -> R {
    if constexpr (SRC)
      return (R)ld_pop(stg + (C * Q + A) * kStageThreads);
    else
      return (R)ld_pop(fc + AA<Q>::template rd<A, PAR>(P, so));
  };
  const R v0 = ldp.template operator()<0>();
  const R g0 = fmx(-(R)L::w(0), fmx(rc[C], P0, dl[C]), v0);
  R d0 = fmx(gkchi, F0, -om * g0);
  R lm[L::NK];
  if constexpr (MRT) {
    refresh();
    R cs[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    R mq[L::NK];
#pragma unroll
    for (int i = 0; i < L::NK; ++i) mq[i] = 0;
    For<0, NP>::run([&]<int K>() {
      constexpr int a = L::pfirst(K), b = L::opp(a);
      V2<R> g;
      R Fe, Fo;
      pair_g(std::integral_constant<int, K>{}, ldp.template operator()<a>(), ldp.template operator()<b>(), g, Fe,
             Fo);
      // {chi Fe + (g_a + g_b), chi Fo + (g_a - g_b)}
      const V2<R> q = fma2(v2(chi, chi), v2(Fe, Fo), add2(v2(g.x, g.x), v2(g.y, -g.y)));
      cs[pclass<Q>(K)] += q.x;
      const R qm = q.y;
      For<0, L::NK>::run([&]<int I>() {
        constexpr int k = L::krow(I);
        constexpr int c = L::m(k, a);
        if constexpr (row_parity<Q>(k) == -1 && c != 0) mq[I] = fmx((R)c, qm, mq[I]);
      });
    });
    // lam_k (M q)_k over the free rows k
    const R q0 = fmx((R)0.5 * chi, F0, g0);
    For<0, L::NK>::run([&]<int I>() {
      constexpr int k = L::krow(I);
      R m = mq[I];
      if constexpr (row_parity<Q>(k) == 1) {
        if constexpr (L::m(k, 0) != 0) m = fmx((R)L::m(k, 0), q0, m);
        For<1, 8>::run([&]<int CL>() {
          if constexpr (crep<Q>(CL) >= 0) {
            constexpr int c = L::m(k, L::pfirst(crep<Q>(CL)));
            if constexpr (c != 0) m = fmx((R)c, cs[CL], m);
          }
        });
      }
      lm[I] = PC<R>::lam(P, I) * m;
    });
    For<0, L::NK>::run([&]<int I>() {
      constexpr int k = L::krow(I);
      if constexpr (row_parity<Q>(k) == 1 && L::m(k, 0) != 0) d0 = fmx(-(R)L::m(k, 0), lm[I], d0);
    });
    asm volatile("" ::: "memory");  // re-read the populations rather than keep them
  }
  // BGK + Guo (+ the MRT correction d_a -= sum_k M_ka lam_k (M q)_k: even part per pair
  // class, odd part per pair), one rounding per stored population
  R rest = dl[C];
  refresh();
  // Pairs in groups of G: the group's loads are issued before its first store. A warp issues
  // in order and the loads stay behind earlier stores, so pair by pair every pair would wait
  // for its own load; a group waits once. Each pair writes exactly the slots it reads (both
  // steps of the AA pattern), so no store of a group touches a slot another pair reads.
  constexpr int G = LBM_COLLIDE_GROUP < NP ? LBM_COLLIDE_GROUP : NP;
  For<0, (NP + G - 1) / G>::run([&]<int GI>() {
    R va[G], vb[G];
    For<0, G>::run([&]<int J>() {
      constexpr int K = GI * G + J;
      if constexpr (K < NP) {
        constexpr int a = L::pfirst(K), b = L::opp(a);
        va[J] = ldp.template operator()<a>();
        vb[J] = ldp.template operator()<b>();
      }
    });
    For<0, G>::run([&]<int J>() {
      constexpr int K = GI * G + J;
      if constexpr (K < NP) {
        constexpr int a = L::pfirst(K), b = L::opp(a);
        V2<R> g;
        R Fe, Fo;
        pair_g(std::integral_constant<int, K>{}, va[J], vb[J], g, Fe, Fo);
        // d = gk chi (Fe +- Fo) - omega g
        V2<R> d = fma2(v2(gkchi, gkchi), add2(v2(Fe, Fe), v2(Fo, -Fo)), mul2(v2(-om, -om), g));
        if constexpr (MRT) {
          R ev = 0, od = 0;
          For<0, L::NK>::run([&]<int I>() {
            constexpr int k = L::krow(I);
            constexpr int c = L::m(k, a);
            if constexpr (c != 0) {
              if constexpr (row_parity<Q>(k) == 1)
                ev = fmx((R)c, lm[I], ev);
              else
                od = fmx((R)c, lm[I], od);
            }
          });
          // d_a - (ev + od), d_b - (ev - od): the sums negated exactly
          d = add2(d, add2(v2(-ev, -ev), v2(-od, od)));
        }
        const V2<R> o = add2(v2(va[J], vb[J]), d);
        const R oa = o.x, ob = o.y;
        if constexpr (sizeof(R) == 4) rest -= oa + ob;
        store_pop<Prec, GLOBAL>(fcw + AA<Q>::template wr<a, PAR>(P, so), oa);
        store_pop<Prec, GLOBAL>(fcw + AA<Q>::template wr<b, PAR>(P, so), ob);
      }
    });
  });
  // The weights rounded to FP32 sum to 1 + 7.5e-9 (D2Q9) or 1 + 1.5e-8 (D3Q19), which makes
  // every step scale the stored deviation rho_c - rho_ref_c by 1 + omega * that excess: a
  // systematic drift of mass from vapour to liquid. The collision conserves each component's
  // mass (the mass row is not relaxed and sum_a Fb_a = 0), so in FP32 the rest population is
  // set from that invariant instead, leaving only unbiased rounding.
  const R out0 = sizeof(R) == 4 ? rest : v0 + d0;
  store_pop<Prec, GLOBAL>(fcw + AA<Q>::template wr<0, PAR>(P, s), out0);
}

// S4-S6 of one site given psi at the site (pn[0]) and its Q - 1 neighbours (pn[a] at x + e_a)
// and the site's moments: total force, split, Guo-forced BGK or MRT collision, in-place AA
// write. Everything is arranged over the pairs of opposite directions (a, b = opp(a)):
//   * the equilibrium is w_a (dl_c + rho_c P_a) with P_a = Pe +- Po (even / odd parts of
//     3 e.u + 9/2 (e.u)^2 - 3/2 u.u); its large even part w (dl_c + rho_c Pe) is the same for
//     both members and is subtracted from each population inside a multiply-add, never
//     rounded on its own;
//   * the Guo term Fb_a = w_a [3 (e_a - u).F + 9 (e_a.u)(e_a.F)] = Fe +- Fo likewise;
//   * the MRT correction acts on the free rows through pair sums (even rows, one coefficient
//     per pair class) and pair differences (odd rows);
//   * the change d_a of each population is formed in full before it is added to the stored
//     value, so the population is rounded once.
// In FP32 these keep the rounding of the large quantities out of the momentum balance; a
// textbook per-direction evaluation lets that rounding drive a random walk of the total
// momentum, and long runs of a liquid slab then drift measurably.
template <int Q, int NC, class Prec, int MRT, int PAR, int GLOBAL = 1, int PT = LBM_COLLIDE_PAIRS, int SRC = 0>
__device__ __forceinline__ void site_collide_m(const Params& P, typename Prec::S* __restrict__ f, const Site& s,
                                               const typename Prec::R (&pn)[Q], const typename Prec::R (&dl)[NC],
                                               const typename Prec::R (&j)[3], typename Prec::S* fo = nullptr,
                                               const float* stg = nullptr) {
  SitePrep<Q, NC, typename Prec::R, PT> sp;
  site_prep<Q, NC, Prec, PT>(P, pn, dl, j, sp);
  For<0, NC>::run([&]<int C>() { comp_collide<Q, NC, Prec, MRT, PAR, C, GLOBAL, PT, SRC>(P, f, s, sp, fo, stg); });
}

// S1 and S4-S6 of one site (the moments, then the collision).
template <int Q, int NC, class Prec, int MRT, int PAR, int GLOBAL = 1, int SRC = 0>
__device__ __forceinline__ void site_collide(const Params& P, typename Prec::S* __restrict__ f, const Site& s,
                                             const typename Prec::R (&pn)[Q], typename Prec::S* fo = nullptr,
                                             const float* stg = nullptr) {
  typename Prec::R dl[NC], j[3];
  site_moments<Q, NC, Prec, PAR, SRC>(P, f, s, dl, j, stg);
  site_collide_m<Q, NC, Prec, MRT, PAR, GLOBAL, LBM_COLLIDE_PAIRS, SRC>(P, f, s, pn, dl, j, fo, stg);
}

// ---------------------------------------------------------------------------------------
// Two-kernel step.

// Pass 1: S1-S3 of every site. Grid (x blocks, y, z), one site per thread.
template <int Q, int NC, class Prec, int PAR>
__device__ __forceinline__ void psi_body(const Params& P, const typename Prec::S* __restrict__ f,
                                         typename Prec::PsiT* __restrict__ psi, int* status, int x) {
  Site s;
  s.set_xyz(P, x, blockIdx.y, blockIdx.z);
  typename Prec::PsiT v;
  const int e = site_psi<Q, NC, Prec, PAR>(P, f, s, v);
  if (e) {
    atomicOr(status, e);
    return;
  }
  psi[s.idx] = v;
}

template <int Q, int NC, class Prec>
__global__ void __launch_bounds__(kBlock) k_psi(const __grid_constant__ Params P, const typename Prec::S* __restrict__ f,
                                                typename Prec::PsiT* __restrict__ psi, int* status,
                                                int parity) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= P.nx) return;
  if (*(volatile int*)status) return;
  if (parity)
    psi_body<Q, NC, Prec, 1>(P, f, psi, status, x);
  else
    psi_body<Q, NC, Prec, 0>(P, f, psi, status, x);
}

// LBM_PSI_VEC4 = 1: the FP32-shifted pseudo-potential pass with 128-bit loads, four consecutive
// x sites per thread (nx divisible by 4). A slot run of four sites starts on a 16-byte boundary
// for every direction at even steps and for the directions without an x component at odd steps
// (one float4 load each); the x-shifted runs of odd steps are loaded site by site. Each site's
// densities are summed in site_densities' order, so psi is bit-identical to k_psi's.
#ifndef LBM_PSI_VEC4
#define LBM_PSI_VEC4 0
#endif
template <int Q, int NC, class Prec, int PAR>
__device__ __forceinline__ void psi4_body(const Params& P, const float* __restrict__ f, float* __restrict__ psi,
                                          int* status, int x4) {
  using L = Lat<Q>;
  Site s;
  s.set_xyz(P, x4, blockIdx.y, blockIdx.z);
  float d[4][NC];
  For<0, NC>::run([&]<int C>() {
    const float* fc = comp_base<Q>(f, P, C);
    float v[Q][4];
    For<0, Q>::run([&]<int A>() {
      constexpr int ex = L::e(A, 0);
      if constexpr (PAR == 0 || ex == 0) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(fc + AA<Q>::template rd<A, PAR>(P, s)));
        v[A][0] = q.x;
        v[A][1] = q.y;
        v[A][2] = q.z;
        v[A][3] = q.w;
      } else {
        // slot (x - e_a, opp a): the run x4 - ex .. x4 + 3 - ex of the row, wrapped at its ends
        constexpr int O = L::opp(A);
        const uint32_t row = s.nb(P, 0, -L::e(A, 1), -L::e(A, 2)) - (uint32_t)x4;
        const float* r = fc + (size_t)O * P.N + row;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          int xx = x4 + k - ex;
          xx = xx < 0 ? xx + P.nx : (xx >= P.nx ? xx - P.nx : xx);
          v[A][k] = __ldg(r + xx);
        }
      }
    });
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float acc = v[0][k];
      For<0, L::NPAIR>::run([&]<int K>() {
        constexpr int a = L::pfirst(K), b = L::opp(a);
        acc += v[a][k] + v[b][k];
      });
      d[k][C] = acc;
    }
  });
  float out[4];
  int err = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float pv;
    err |= site_psi_dl<NC, Prec>(P, d[k], pv);
    out[k] = pv;
  }
  if (err) {
    atomicOr(status, err);
    return;
  }
  *reinterpret_cast<float4*>(psi + s.idx) = make_float4(out[0], out[1], out[2], out[3]);
}
template <int Q, int NC, class Prec>
__global__ void __launch_bounds__(kBlock) k_psi4(const __grid_constant__ Params P, const float* __restrict__ f,
                                                 float* __restrict__ psi, int* status, int parity) {
  const int x4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (x4 >= P.nx) return;
  if (*(volatile int*)status) return;
  if (parity)
    psi4_body<Q, NC, Prec, 1>(P, f, psi, status, x4);
  else
    psi4_body<Q, NC, Prec, 0>(P, f, psi, status, x4);
}

// Pass 2: S4-S6 of every site; psi of the neighbours from global memory.
template <int Q, int NC, class Prec, int MRT, int PAR, int GLOBAL = 1, int SRC = 0>
__device__ __forceinline__ void collide_site(const Params& P, typename Prec::S* __restrict__ f,
                                             const typename Prec::PsiT* __restrict__ psi, int x, int y, int z,
                                             typename Prec::S* fo, const float* stg = nullptr) {
  using R = typename Prec::R;
  using L = Lat<Q>;
  Site s;
  s.set_xyz(P, x, y, z);
  R pn[Q];
  pn[0] = (R)psi[s.idx];
#pragma unroll
  for (int a = 1; a < Q; ++a) pn[a] = (R)psi[s.nb(P, L::e(a, 0), L::e(a, 1), L::e(a, 2))];
  site_collide<Q, NC, Prec, MRT, PAR, GLOBAL, SRC>(P, f, s, pn, fo, stg);
}
template <int Q, int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void collide_body(const Params& P, typename Prec::S* __restrict__ f,
                                             const typename Prec::PsiT* __restrict__ psi, int x,
                                             typename Prec::S* fo = nullptr) {
  collide_site<Q, NC, Prec, MRT, PAR>(P, f, psi, x, blockIdx.y, blockIdx.z, fo);
}

// LBM_COLLIDE_PSI_SMEM = 1: the block first stages the pseudo-potential its sites' stencils
// need in shared memory (the rows (y + dy, z + dz) around its row segment, one site of halo at
// each x end, coalesced loads), then every site reads its 19 values from there; 0 (the default,
// faster on GB300, see the design notes): each site loads them from global memory (L1 / L2).
#ifndef LBM_COLLIDE_PSI_SMEM
#define LBM_COLLIDE_PSI_SMEM 0
#endif
template <int Q, int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void collide_body_smem(const Params& P, typename Prec::S* __restrict__ f,
                                                  const typename Prec::PsiT* __restrict__ psi) {
  using R = typename Prec::R;
  using PsiT = typename Prec::PsiT;
  using L = Lat<Q>;
  constexpr int NR = Q == 19 ? 9 : 3;  // rows (dy, dz) of the stencil
  __shared__ PsiT sp[NR][kCollideThreads + 2];
  const int bx = blockDim.x, x0 = blockIdx.x * bx, y = blockIdx.y, z = blockIdx.z;
  const int w = min(bx, P.nx - x0) + 2;
  for (int r = 0; r < NR; ++r) {
    const int dy = r / 3 - 1, dz = Q == 19 ? r % 3 - 1 : 0;
    const int yy = dy == 0 ? y : (dy > 0 ? (y == P.ny - 1 ? 0 : y + 1) : (y == 0 ? P.ny - 1 : y - 1));
    const int zz = dz == 0 ? z : (dz > 0 ? (z == P.nz - 1 ? 0 : z + 1) : (z == 0 ? P.nz - 1 : z - 1));
    const PsiT* row = psi + ((size_t)zz * P.ny + yy) * P.nx;
    for (int i = threadIdx.x; i < w; i += bx) {
      int xx = x0 - 1 + i;
      xx = xx < 0 ? xx + P.nx : (xx >= P.nx ? xx - P.nx : xx);
      sp[r][i] = row[xx];
    }
  }
  __syncthreads();
  const int x = x0 + threadIdx.x;
  if (x >= P.nx) return;
  R pn[Q];
  For<0, Q>::run([&]<int A>() {
    constexpr int r = (L::e(A, 1) + 1) * 3 + (Q == 19 ? L::e(A, 2) + 1 : 0);
    pn[A] = (R)sp[Q == 19 ? r : L::e(A, 1) + 1][threadIdx.x + 1 + L::e(A, 0)];
  });
  Site s;
  s.set_xyz(P, x, y, z);
  site_collide<Q, NC, Prec, MRT, PAR>(P, f, s, pn);
}

template <int Q, int NC, class Prec, int MRT>
__global__ void __launch_bounds__(kCollideThreads, kCollideBlocksOf<Q, Prec>) k_collide(const __grid_constant__ Params P, typename Prec::S* __restrict__ f,
                                                       const typename Prec::PsiT* __restrict__ psi,
                                                       const int* status, long long* t_dev, int parity) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (*(volatile const int*)status) return;
  // the step counter advances only for steps whose pseudo-potential pass succeeded
  if (x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *t_dev += 1;
  if constexpr (LBM_COLLIDE_PSI_SMEM) {
    if (parity)
      collide_body_smem<Q, NC, Prec, MRT, 1>(P, f, psi);
    else
      collide_body_smem<Q, NC, Prec, MRT, 0>(P, f, psi);
    return;
  }
  if (x >= P.nx) return;
  if (parity)
    collide_body<Q, NC, Prec, MRT, 1>(P, f, psi, x);
  else
    collide_body<Q, NC, Prec, MRT, 0>(P, f, psi, x);
}

// LBM_COLLIDE_STAGED = 1 (FP32-shifted storage): the collide pass as a persistent loop over
// row segments of kStageThreads sites. Each thread copies the populations of its site in the
// next segment into shared memory (cp.async, 4 bytes each: the copies hold no registers and
// their latency runs under the current site's collision) and computes the current site from
// its own staged copy, so the DRAM latency of a site's 57 loads is off its critical path.
// Each thread reads only what it copied itself: no block barrier. The slots of the next site
// are disjoint from those the current site writes (every site reads and writes its own set),
// so the early copy reads values no one writes in this step. Two stages of NC Q kStageThreads
// floats per block. Measured on GB300 (256^3 sphere workload, bit-identical states): 1.72 ms per
// collide pass against 1.50 ms for k_collide, so it is off. It removes half of the DRAM-latency
// stalls but its shared memory (29 KB per 64-thread block, two stages) caps the SM at 12 warps
// against k_collide's 14.5, and the carve-out leaves L1 too little room for the
// pseudo-potential stencil.
#ifndef LBM_COLLIDE_STAGED
#define LBM_COLLIDE_STAGED 0
#endif
#ifndef LBM_COLLIDE_STAGED_BLOCKS
#define LBM_COLLIDE_STAGED_BLOCKS 6  // 170 registers, no spills; 12 warps per SM
#endif
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int Q, int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void collide_staged_body(const Params& P, float* __restrict__ f,
                                                    const float* __restrict__ psi) {
  extern __shared__ float stage_sm[];
  constexpr int T = kStageThreads, STAGE = NC * Q * T;
  const int tid = threadIdx.x;
  // items (segment, y, z), segment fastest; nseg ny nz <= N < 2^32 / Q fits an int. A block
  // takes items blockIdx.x, + gridDim.x, ...: the coordinates advance by the mixed-radix digits
  // of gridDim.x (no division per item)
  const int nseg = (P.nx + T - 1) / T;
  const int nitems = nseg * P.ny * P.nz;
  const int G = (int)gridDim.x, gs = G % nseg, gy = (G / nseg) % P.ny, gz = G / nseg / P.ny;
  auto advance = [&](int& sg, int& yy, int& zz) {
    sg += gs;
    int c = sg >= nseg;
    sg -= c ? nseg : 0;
    yy += gy + c;
    c = yy >= P.ny;
    yy -= c ? P.ny : 0;
    zz += gz + c;
  };
  // copies of the site (seg, y, z) of this thread, if it has one, into stage buf
  auto issue = [&](int sg, int yy, int zz, int buf) -> bool {
    const int x = sg * T + tid;
    if (x >= P.nx) return false;
    Site s;
    s.set_xyz(P, x, yy, zz);
    float* dst = stage_sm + buf * STAGE + tid;
    For<0, NC>::run([&]<int C>() {
      const float* fc = comp_base<Q>((const float*)f, P, C);
      For<0, Q>::run([&]<int A>() { cp_async4(dst + (C * Q + A) * T, fc + AA<Q>::template rd<A, PAR>(P, s)); });
    });
    return true;
  };
  int item = (int)blockIdx.x;
  int seg = item % nseg, y = (item / nseg) % P.ny, z = item / nseg / P.ny;
  int buf = 0;
  bool have = item < nitems && issue(seg, y, z, 0);
  cp_async_commit();
  while (item < nitems) {
    const int nxt = item + G;
    int sn = seg, yn = y, zn = z;
    advance(sn, yn, zn);
    const bool have_n = nxt < nitems && issue(sn, yn, zn, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of the current item have landed
    if (have)
      collide_site<Q, NC, Prec, MRT, PAR, 1, 1>(P, f, psi, seg * T + tid, y, z, nullptr, stage_sm + buf * STAGE + tid);
    item = nxt;
    seg = sn;
    y = yn;
    z = zn;
    have = have_n;
    buf ^= 1;
  }
  cp_async_wait<0>();
}

template <int Q, int NC, class Prec, int MRT>
__global__ void __launch_bounds__(kStageThreads, LBM_COLLIDE_STAGED_BLOCKS)
    k_collide_staged(const __grid_constant__ Params P, float* __restrict__ f, const float* __restrict__ psi,
                     const int* status, long long* t_dev, int parity) {
  if (*(volatile const int*)status) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *t_dev += 1;
  if (parity)
    collide_staged_body<Q, NC, Prec, MRT, 1>(P, f, psi);
  else
    collide_staged_body<Q, NC, Prec, MRT, 0>(P, f, psi);
}

// The collide pass out of place: reads the state in fin, writes the next one to fout (the
// adjoint's replay keeps every state of a segment; the AA pattern makes the two buffers hold
// the same slots, so fout needs no copy of fin first).
template <int Q, int NC, class Prec, int MRT>
__global__ void __launch_bounds__(kCollideThreads, kCollideBlocksOf<Q, Prec>)
    k_collide_oop(const __grid_constant__ Params P, typename Prec::S* __restrict__ fin, typename Prec::S* __restrict__ fout,
                  const typename Prec::PsiT* __restrict__ psi, const int* status, long long* t_dev, int parity) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= P.nx) return;
  if (*(volatile const int*)status) return;
  if (x == 0 && blockIdx.y == 0 && blockIdx.z == 0) *t_dev += 1;
  if (parity)
    collide_body<Q, NC, Prec, MRT, 1>(P, fin, psi, x, fout);
  else
    collide_body<Q, NC, Prec, MRT, 0>(P, fin, psi, x, fout);
}

// ---------------------------------------------------------------------------------------
// Fused step.
// Compile-time options of the fused step: planes per synchronisation round, the psi stencil
// from a shared-memory window (1) or straight from L2 (0), and an L2 prefetch of the
// populations the next round's psi stage reads (1).
#ifndef LBM_FUSED_P
#define LBM_FUSED_P 4
#endif
#ifndef LBM_FUSED_WINDOW
#define LBM_FUSED_WINDOW 0
#endif
#ifndef LBM_FUSED_PREFETCH
#define LBM_FUSED_PREFETCH 0
#endif

template <int Q>
struct Fused;
template <>
struct Fused<19> {  // tile of 32 x 8 sites in (x, y), march along z
  static constexpr int TX = 32, TY = 8, NT = TX * TY, WY = TY + 2, P = LBM_FUSED_P;
};
template <>
struct Fused<9> {  // tile of 128 sites in x, march along y
  static constexpr int TX = 128, TY = 1, NT = TX, WY = 1, P = LBM_FUSED_P;
};

struct FusedArgs {
  unsigned long long* flags;  // one progress counter per block (stages published)
  unsigned int* done;         // blocks finished in the current launch
  int* pending;               // status bits raised in the current launch
  int ntx, nty, nchunk, L;    // tiles along x and y (1 in 2-D), chunks and chunk length
  int silent_block;           // test hook: this block publishes no progress (-1: none)
  // plane-range form (k_fused3, D3Q19)
  int mode;                   // 1 (or 0): tile columns (k_fused), 3: plane ranges (k_fused3),
                              // 4: plane ranges with trailing psi (k_trail3),
                              // 5: task queue with trailing psi (k_trailq)
  const int* range;           // G + 1 range starts in the flattened (y, x) index of a plane
  const int* nbr;             // G x kF3MaxNbr workers owning neighbour sites, -1 padded
                              // (k_trailq: nch x kF3MaxNbr chunks)
  void* psi_ring;             // k_fused3: (kF3Ring + 2) psi planes; k_trail3, k_trailq: two psi fields
  int G, smax;                // workers (two per CTA), largest range; k_trailq: CTAs, sites per chunk
  // task-queue form (k_trailq, mode 5): the ticket order of the step's tasks (collision of
  // chunk c of plane z: z nch + c; psi of the next step there: -(z nch + c) - 1), the ticket
  // counter, chunks per plane
  const int* tasks;
  int ntask, nch;
  unsigned int* ticket;
};

constexpr unsigned kSpinLimit = 1u << 20;  // polls of one flag before giving up (~1 s)

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// One launch = one time step. Block b owns tile (tx, ty) of chunk ch: planes [p0, p0 + L) of
// the march axis (z for D3Q19, y for D2Q9), in G = L / P groups of P planes. Stage s computes
// psi of one group and publishes it (progress counter = base + s + 1): stage 0 is the chunk's
// last group (needed first by the chunk above), stage s >= 1 is group s - 1. Colliding group j
// needs psi of the plane below and above the group, from this and the neighbouring tiles, so
// it waits for the neighbours' counters to reach min(j + 3, G) (the chunk below's last group
// for j = 0, the chunk above's first group for j = G - 1). Iteration j first computes stage
// j + 2 (group j + 1), then waits, then collides group j: a stage never waits within its own
// iteration and every wait refers to stages the neighbours compute before their own wait of
// the same iteration, so with all blocks co-resident the pipeline cannot deadlock (and every
// wait is bounded anyway). Group j + 1 is read for its psi one iteration before it is
// collided, and its populations are meant to be re-read from L2: between the two reads the
// grid touches about three groups of planes (the collision of group j - 1, reads and writes,
// and the psi of group j + 1), 45 MB per plane group for 256^2 sites and 3 FP32 D3Q19
// components, so one plane per group keeps the re-read inside the 129 MB L2.
template <int Q, int NC, class Prec, int MRT, int PAR>
__device__ __forceinline__ void fused_body(const Params& P, typename Prec::S* __restrict__ f,
                                           typename Prec::PsiT* __restrict__ psi_g, int* status, long long* t_dev,
                                           const FusedArgs& A, unsigned long long t) {
  using Gm = Fused<Q>;
  using R = typename Prec::R;
  using PsiT = typename Prec::PsiT;
  using L = Lat<Q>;
  constexpr bool D3 = Q == 19;
  constexpr int TX = Gm::TX, TY = Gm::TY, WY = Gm::WY, WX = TX + 2, NP = Gm::P, NS = NP + 2;
  __shared__ PsiT win[NS][WY][WX];
  __shared__ int nbr[27];
  __shared__ int nbr_need[27];  // 0 = same chunk, 1 = chunk below, 2 = chunk above
  __shared__ int n_nbr;

  const int L_ = A.L, G = A.L / NP;
  const unsigned long long base = t * (unsigned long long)G;
  const int b = blockIdx.x;
  const int tx = b % A.ntx;
  const int ty = (b / A.ntx) % A.nty;
  const int ch = b / (A.ntx * A.nty);
  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int cx = tx * TX + lx;
  const int cy = D3 ? ty * TY + ly : 0;
  const int nm = D3 ? P.nz : P.ny;
  const int p0 = ch * L_;

  if (threadIdx.x == 0) {
    int n = 0;
    for (int kind = 0; kind < 3; ++kind) {
      int cc = kind == 0 ? ch : (kind == 1 ? (ch + A.nchunk - 1) % A.nchunk : (ch + 1) % A.nchunk);
      for (int dy = D3 ? -1 : 0; dy <= (D3 ? 1 : 0); ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (kind == 0 && dx == 0 && dy == 0) continue;
          int ttx = (tx + dx + A.ntx) % A.ntx, tty = (ty + dy + A.nty) % A.nty;
          nbr[n] = (cc * A.nty + tty) * A.ntx + ttx;
          nbr_need[n] = kind;
          ++n;
        }
    }
    n_nbr = n;
  }

  auto site_at = [&](int m, Site& st) {
    if constexpr (D3)
      st.set_xyz(P, cx, cy, m);
    else
      st.set_xyz(P, cx, m, 0);
  };
  int err = 0;
  // stage s: psi of the NP planes of group (s == 0 ? G - 1 : s - 1)
  auto stage = [&](int s_) {
    const int g = s_ == 0 ? G - 1 : s_ - 1;
    PsiT v[NP];
    uint32_t ix[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      Site st;
      site_at(p0 + g * NP + i, st);
      ix[i] = st.idx;
      err |= site_psi<Q, NC, Prec, PAR>(P, f, st, v[i]);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) psi_g[ix[i]] = v[i];
    __syncthreads();
    if (threadIdx.x == 0 && b != A.silent_block) st_release_u64(&A.flags[b], base + (unsigned long long)(s_ + 1));
  };
  bool ok = true;
  // waits until every neighbour of the selected kind has published `need` stages
  auto wait = [&](int kind, int need) {
    bool mine = true;
    if (ok && threadIdx.x < n_nbr && nbr_need[threadIdx.x] == kind) {
      const unsigned long long target = base + (unsigned long long)need;
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
  // psi of plane p0 + q (q may be -1 or L: the neighbouring chunks) into its ring slot, through
  // L2 (written by other blocks)
  auto load_plane = [&](int q) {
    const int gm = ((p0 + q) % nm + nm) % nm;
    const int slot = (q + 1 + NS) % NS;
    for (int i = threadIdx.x; i < WY * WX; i += Gm::NT) {
      const int wx = i % WX, wy = i / WX;
      const int gx = (tx * TX + wx - 1 + P.nx) % P.nx;
      const int gy = D3 ? (ty * TY + wy - 1 + P.ny) % P.ny : 0;
      const int64_t idx = D3 ? ((int64_t)gm * P.ny + gy) * P.nx + gx : (int64_t)gm * P.nx + gx;
      win[slot][wy][wx] = __ldcg(psi_g + idx);
    }
  };

  __syncthreads();  // neighbour list ready
  stage(0);
  stage(1);
  if (G > 2) stage(2);
  wait(1, 1);  // chunk below: its last group (plane p0 - 1)
  wait(0, 2);  // this chunk's tiles: group 0 (plane p0)
  if (LBM_FUSED_WINDOW && ok) {
    load_plane(-1);
    load_plane(0);
  }
  for (int j = 0; j < G && ok; ++j) {
    if (j >= 1 && j + 2 < G) stage(j + 2);
    // planes p0 + jP + 1 .. p0 + jP + NP: groups j and j + 1 of this chunk, or the chunk
    // above's first group for the last group
    wait(0, j + 3 < G ? j + 3 : G);
    if (j == G - 1) wait(2, 2);
    if (!ok) break;
    if constexpr (LBM_FUSED_PREFETCH) {
      // the populations of group j + 2 (next round's psi stage) into L2
      if (j + 2 < G) {
#pragma unroll 1
        for (int i = 0; i < NP; ++i) {
          Site st;
          site_at(p0 + (j + 2) * NP + i, st);
          For<0, NC>::run([&]<int C>() {
            const typename Prec::S* fc = comp_base<Q>(f, P, C);
            For<0, Q>::run([&]<int A>() {
              asm volatile("prefetch.global.L2 [%0];" ::"l"(fc + AA<Q>::template rd<A, PAR>(P, st)));
            });
          });
        }
      }
    }
    if constexpr (LBM_FUSED_WINDOW) {
      for (int i = 1; i <= NP; ++i) load_plane(j * NP + i);
      __syncthreads();
    }
#pragma unroll 1
    for (int i = 0; i < NP; ++i) {
      const int q = j * NP + i;
      Site st;
      site_at(p0 + q, st);
      R pn[Q];
      if constexpr (LBM_FUSED_WINDOW) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const int em = D3 ? L::e(a, 2) : L::e(a, 1);
          const int ey = D3 ? L::e(a, 1) : 0;
          pn[a] = (R)win[(q + 1 + em + NS) % NS][D3 ? ly + 1 + ey : 0][lx + 1 + L::e(a, 0)];
        }
      } else {
        pn[0] = (R)__ldcg(psi_g + st.idx);
#pragma unroll
        for (int a = 1; a < Q; ++a) pn[a] = (R)__ldcg(psi_g + st.nb(P, L::e(a, 0), L::e(a, 1), L::e(a, 2)));
      }
      site_collide<Q, NC, Prec, MRT, PAR>(P, f, st, pn);
    }
  }
  if (!ok) err |= ST_TIMEOUT;
  // finish: the last block of the launch folds the pending status and advances the step
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

template <int Q, int NC, class Prec, int MRT>
__global__ void __launch_bounds__(Fused<Q>::NT, Q == 19 ? 2 : 4)
    k_fused(const Params P, typename Prec::S* __restrict__ f, typename Prec::PsiT* __restrict__ psi_g, int* status,
            long long* t_dev, const FusedArgs A) {
  if (*(volatile int*)status) return;  // a previous step failed: do nothing
  const unsigned long long t = (unsigned long long)*(volatile long long*)t_dev;
  if (t & 1)
    fused_body<Q, NC, Prec, MRT, 1>(P, f, psi_g, status, t_dev, A, t);
  else
    fused_body<Q, NC, Prec, MRT, 0>(P, f, psi_g, status, t_dev, A, t);
}

// ---------------------------------------------------------------------------------------
// Set-up and read-back kernels (FP64 arithmetic, not on the timed path).

// f = f_eq(rho_c, u) of Eq. equilibrium(a), stored in the even layout, shift subtracted:
// f - w_a rho_ref = w_a [(rho - rho_ref) + rho P_a], P_a = 3 e.u + 9/2 (e.u)^2 - 3/2 u.u. The
// difference rho - rho_ref is taken in FP64; for FP32 storage the rest is FP32 arithmetic
// (its result is rounded to FP32 anyway), for FP64 storage FP64.
template <int Q, int NC, class Prec>
__global__ void k_init(const Params P, typename Prec::S* f, const double* __restrict__ rho,
                       const double* __restrict__ u) {
  using L = Lat<Q>;
  using R = typename Prec::R;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  R uv[3] = {0, 0, 0}, uu = 0;
  if (u) {
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
      uv[d] = (R)u[d * P.N + idx];
      uu += uv[d] * uv[d];
    }
  }
  R pa[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    R eu = 0;
#pragma unroll
    for (int d = 0; d < L::D; ++d) {
      if (L::e(a, d) > 0) eu += uv[d];
      if (L::e(a, d) < 0) eu -= uv[d];
    }
    pa[a] = eu * ((R)3 + (R)4.5 * eu) - (R)1.5 * uu;
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double r = rho[c * P.N + idx];
    const R dr = (R)(r - P.rho_ref[c]);
    const R rr = (R)r;
#pragma unroll
    for (int a = 0; a < Q; ++a)
      f[((int64_t)c * Q + a) * P.N + idx] = (typename Prec::S)((R)L::w(a) * (dr + rr * pa[a]));
  }
}

// canonical FP64 populations <-> storage
template <int Q, int NC, class Prec, int PAR>
__device__ __forceinline__ void get_f_body(const Params& P, const typename Prec::S* __restrict__ f, double* out,
                                           const Site& s) {
  For<0, NC>::run([&]<int C>() {
    const typename Prec::S* fc = comp_base<Q>(f, P, C);
    For<0, Q>::run([&]<int A>() {
      out[((int64_t)C * Q + A) * P.N + s.idx] = (double)fc[AA<Q>::template rd<A, PAR>(P, s)] + Lat<Q>::w(A) * P.rho_ref[C];
    });
  });
}

template <int Q, int NC, class Prec>
__global__ void k_get_f(const Params P, const typename Prec::S* __restrict__ f, double* out, int parity) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  Site s;
  s.set(P, (uint32_t)idx);
  if (parity)
    get_f_body<Q, NC, Prec, 1>(P, f, out, s);
  else
    get_f_body<Q, NC, Prec, 0>(P, f, out, s);
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

// Macroscopic fields of the current state: component densities, barycentric velocity with the
// Guo half force, EOS pressure and psi; each only when its output pointer is set (psi must hold
// this state's pseudo-potential when u or psi is asked for). Moments and force in the storage
// precision's arithmetic, the EOS in FP64, outputs FP64.
template <int Q, int NC, class Prec, int PAR>
__device__ __forceinline__ void fields_body(const Params& P, const typename Prec::S* __restrict__ f,
                                            const typename Prec::PsiT* __restrict__ psi, double* rho_out,
                                            double* u_out, double* p_out, double* psi_out, const Site& s) {
  using L = Lat<Q>;
  using R = typename Prec::R;
  const int64_t idx = s.idx;
  R dl[NC], j[3];
  site_moments<Q, NC, Prec, PAR>(P, f, s, dl, j);
  double rc[NC], rho = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    rc[c] = P.rho_ref[c] + (double)dl[c];
    rho += rc[c];
    if (rho_out) rho_out[c * P.N + idx] = rc[c];
  }
  if (u_out) {
    R s1[3] = {0, 0, 0}, s2[3] = {0, 0, 0};
    For<1, Q>::run([&]<int A>() {
      const R pn = (R)psi[s.nb(P, L::e(A, 0), L::e(A, 1), L::e(A, 2))];
#pragma unroll
      for (int d = 0; d < L::D; ++d) {
        if (L::e(A, d) != 0) {
          s1[d] += (R)(L::w(A) * L::e(A, d)) * pn;
          s2[d] += (R)(L::w(A) * L::e(A, d)) * pn * pn;
        }
      }
    });
    const R p0 = (R)psi[idx];
    for (int d = 0; d < 3; ++d) {
      const R F = d < L::D ? PC<R>::c1(P) * p0 * s1[d] + PC<R>::c2(P) * s2[d] : (R)0;
      u_out[d * P.N + idx] = (double)((j[d] + (R)0.5 * F) / (R)rho);
    }
  }
  if (p_out) {
    EosOut<NC> e = eos_pr<NC>(P, rc);
    p_out[idx] = e.pD / e.Dd;
  }
  if (psi_out) psi_out[idx] = (double)psi[idx];
}

template <int Q, int NC, class Prec>
__global__ void k_fields(const Params P, const typename Prec::S* __restrict__ f,
                         const typename Prec::PsiT* __restrict__ psi, double* rho_out, double* u_out,
                         double* p_out, double* psi_out, int parity) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P.N) return;
  Site s;
  s.set(P, (uint32_t)idx);
  if (parity)
    fields_body<Q, NC, Prec, 1>(P, f, psi, rho_out, u_out, p_out, psi_out, s);
  else
    fields_body<Q, NC, Prec, 0>(P, f, psi, rho_out, u_out, p_out, psi_out, s);
}

// S7 per-component mass M_c = sum over sites and slots of the stored value, plus N rho_ref_c
// (every slot of a component holds exactly one population in either AA layout, and the
// shifts w_a rho_ref_c of one site's slots add up to rho_ref_c since sum_a w_a = 1; the
// N rho_ref_c term is added once by k_mass_final). FP32 populations are summed per thread
// with Knuth's TwoSum: a compensated FP32 sum, about 2^-48 relative, on the FP32 pipe (a
// per-population conversion to FP64 would run on GB300's 1/64-rate FP64 pipe); FP64
// populations are summed in FP64. Threads walk the sites with the fixed stride of a fixed grid
// (kMassBlocks), and the blocks and k_mass_final reduce in FP64 in a fixed order, so the result
// does not depend on scheduling.
constexpr int kMassBlocks = 1024;
template <int Q, int NC, class Prec>
__global__ void __launch_bounds__(kBlock) k_mass_partial(const Params P, const typename Prec::S* __restrict__ f,
                                                         double* partial) {
  __shared__ double sh[kBlock];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int c = 0; c < NC; ++c) {
    const typename Prec::S* fc = f + (int64_t)c * Q * P.N;
    double v = 0;
    if constexpr (sizeof(typename Prec::S) == 4) {
      float hi = 0.f, lo = 0.f;
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += stride) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
          const float x = fc[(int64_t)a * P.N + i];
          const float sm = hi + x;
          const float bp = sm - hi;
          lo += (hi - (sm - bp)) + (x - bp);
          hi = sm;
        }
      }
      v = (double)hi + (double)lo;
    } else {
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.N; i += stride) {
#pragma unroll
        for (int a = 0; a < Q; ++a) v += (double)fc[(int64_t)a * P.N + i];
      }
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

struct MassShift {
  double v[4];  // N rho_ref_c per component
};
__global__ void k_mass_final(const double* partial, int nblocks, int nc, MassShift shift, double* out);

}  // namespace lbm

#include "lbm_fused3.cuh"
#include "lbm_trail3.cuh"
#include "lbm_trailq.cuh"

namespace lbm {

// ---------------------------------------------------------------------------------------
// Host launchers and the dispatch table of one (Q, NC, precision, collision).
template <int Q, int NC, class Prec, int MRT>
struct Launch {
  using S = typename Prec::S;
  using R = typename Prec::R;
  using PsiT = typename Prec::PsiT;
  static unsigned blocks(const Params& P) { return (unsigned)((P.N + kBlock - 1) / kBlock); }
  // resident blocks of kernel k with `threads` threads (32 .. 512) on the whole device, queried
  // once per kernel and block size (0 when the query fails)
  template <class K>
  static int wave_blocks(K k, int threads) {
    static std::atomic<int> cache[5] = {-1, -1, -1, -1, -1};
    int i = 0;
    while (i < 4 && (32 << i) < threads) ++i;
    int w = cache[i].load(std::memory_order_relaxed);
    if (w >= 0) return w;
    int nb = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, 0) != cudaSuccess) {
      cudaGetLastError();
      nb = 0;
    }
    w = nb * sms;
    cache[i].store(w, std::memory_order_relaxed);
    return w;
  }
  // both passes of the two-kernel step fit in one wave of resident blocks each
  static bool single_wave(const Params& P) {
    dim3 g1, b1, g2, b2;
    site_grid(P, g1, b1);
    site_grid(P, g2, b2, kCollideThreads);
    return (long long)g1.x * g1.y * g1.z <= wave_blocks(k_psi<Q, NC, Prec>, (int)b1.x) &&
           (long long)g2.x * g2.y * g2.z <= wave_blocks(k_collide<Q, NC, Prec, MRT>, (int)b2.x);
  }
  // a pass of the two-kernel step, launched as a programmatic dependent of the kernel before it
  // when the step is single-wave (plainly otherwise, when LBM_PDL = 0 or when the attribute is
  // refused)
  template <class... KArgs, class... Args>
  static void launch_pass(void (*k)(KArgs...), bool pdl, dim3 g, dim3 b, cudaStream_t s, Args... args) {
    if (LBM_PDL && pdl) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = g;
      cfg.blockDim = b;
      cfg.dynamicSmemBytes = 0;
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, k, args...) == cudaSuccess) return;
      cudaGetLastError();
    }
    k<<<g, b, 0, s>>>(args...);
  }
  // site grid of the step passes: x in blocks of up to 256 threads, one block row per (y, z)
  static void site_grid(const Params& P, dim3& grid, dim3& block, int maxt = kBlock) {
    int tx = 32;
    while (tx < P.nx && tx < maxt) tx *= 2;
    block = dim3(tx);
    grid = dim3((unsigned)((P.nx + tx - 1) / tx), (unsigned)P.ny, (unsigned)P.nz);
  }
  static void psi(const Params& P, const void* f, void* ps, int* st, int parity, cudaStream_t s) {
    if constexpr (LBM_PSI_VEC4 && std::is_same_v<S, float>) {
      if (P.nx % 4 == 0) {
        int tx = 32;
        while (tx < P.nx / 4 && tx < kBlock) tx *= 2;
        const dim3 g((unsigned)((P.nx / 4 + tx - 1) / tx), (unsigned)P.ny, (unsigned)P.nz);
        k_psi4<Q, NC, Prec><<<g, tx, 0, s>>>(P, (const float*)f, (float*)ps, st, parity);
        return;
      }
    }
    dim3 g, b;
    site_grid(P, g, b);
    launch_pass(k_psi<Q, NC, Prec>, single_wave(P), g, b, s, P, (const S*)f, (PsiT*)ps, st, parity);
  }
  static void collide(const Params& P, void* f, const void* ps, const int* st, long long* t_dev, int parity,
                      cudaStream_t s) {
    if constexpr (LBM_COLLIDE_STAGED && std::is_same_v<S, float> && std::is_same_v<PsiT, float>) {
      static int grid = 0;  // resident blocks of the persistent kernel, set once per process
      constexpr size_t smem = (size_t)2 * NC * Q * kStageThreads * sizeof(float);
      auto k = k_collide_staged<Q, NC, Prec, MRT>;
      if (grid == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, kStageThreads, smem);
        grid = sms * (per > 0 ? per : 1);
      }
      const long long items = (long long)((P.nx + kStageThreads - 1) / kStageThreads) * P.ny * P.nz;
      const int g = (int)std::min<long long>(items, grid);
      k<<<g, kStageThreads, smem, s>>>(P, (float*)f, (const float*)ps, st, t_dev, parity);
      return;
    }
    dim3 g, b;
    site_grid(P, g, b, kCollideThreads);
    launch_pass(k_collide<Q, NC, Prec, MRT>, single_wave(P), g, b, s, P, (S*)f, (const PsiT*)ps, st, t_dev, parity);
  }
  static void collide_oop(const Params& P, const void* fin, void* fout, const void* ps, const int* st,
                          long long* t_dev, int parity, cudaStream_t s) {
    dim3 g, b;
    site_grid(P, g, b, kCollideThreads);
    k_collide_oop<Q, NC, Prec, MRT><<<g, b, 0, s>>>(P, (S*)fin, (S*)fout, (const PsiT*)ps, st, t_dev, parity);
  }
  static int fused_max_blocks() {
    int nb = 0, dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused<Q, NC, Prec, MRT>, Fused<Q>::NT, 0) !=
        cudaSuccess)
      return 0;
    return nb * sms;
  }
  static cudaError_t fused(const Params& P, void* f, void* ps, int* st, long long* t_dev, const FusedArgs& A,
                           cudaStream_t s) {
    S* fp = (S*)f;
    PsiT* pp = (PsiT*)ps;
    Params Pc = P;
    FusedArgs Ac = A;
    void* args[] = {(void*)&Pc, (void*)&fp, (void*)&pp, (void*)&st, (void*)&t_dev, (void*)&Ac};
    const unsigned grid = (unsigned)(A.ntx * A.nty * A.nchunk);
    return cudaLaunchCooperativeKernel((const void*)k_fused<Q, NC, Prec, MRT>, dim3(grid), dim3(Fused<Q>::NT),
                                       args, 0, s);
  }
  static int fused3_max_blocks(int smem) {
    if constexpr (Q != 19) {
      return 0;
    } else {
      int nb = 0, dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess) return 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
      if (cudaFuncSetAttribute(k_fused3<NC, Prec, MRT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
              cudaSuccess ||
          cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fused3<NC, Prec, MRT>, kF3Threads, smem) !=
              cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return nb * sms;
    }
  }
  static cudaError_t fused3(const Params& P, void* f, int* st, long long* t_dev, const FusedArgs& A, cudaStream_t s) {
    if constexpr (Q != 19) {
      return cudaErrorNotSupported;
    } else {
      S* fp = (S*)f;
      Params Pc = P;
      FusedArgs Ac = A;
      void* args[] = {(void*)&Pc, (void*)&fp, (void*)&st, (void*)&t_dev, (void*)&Ac};
      const size_t smem = 0;
      return cudaLaunchCooperativeKernel((const void*)k_fused3<NC, Prec, MRT>, dim3((unsigned)(A.G / kF3WorkersPerCta)),
                                         dim3(kF3Threads), args, smem, s);
    }
  }
  static int trail3_max_blocks() {
    if constexpr (Q != 19) {
      return 0;
    } else {
      int nb = 0, dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess) return 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trail3<NC, Prec, MRT>, kT3Threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return nb * sms;
    }
  }
  static cudaError_t trail3(const Params& P, void* f, int* st, long long* t_dev, const FusedArgs& A, cudaStream_t s) {
    if constexpr (Q != 19) {
      return cudaErrorNotSupported;
    } else {
      S* fp = (S*)f;
      Params Pc = P;
      FusedArgs Ac = A;
      void* args[] = {(void*)&Pc, (void*)&fp, (void*)&st, (void*)&t_dev, (void*)&Ac};
      return cudaLaunchCooperativeKernel((const void*)k_trail3<NC, Prec, MRT>, dim3((unsigned)A.G),
                                         dim3(kT3Threads), args, 0, s);
    }
  }
  static int trailq_max_blocks() {
    if constexpr (Q != 19) {
      return 0;
    } else {
      int nb = 0, dev = 0, sms = 0;
      if (cudaGetDevice(&dev) != cudaSuccess) return 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_trailq<NC, Prec, MRT>, kTQThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return nb * sms;
    }
  }
  static cudaError_t trailq(const Params& P, void* f, int* st, long long* t_dev, const FusedArgs& A, cudaStream_t s) {
    if constexpr (Q != 19) {
      return cudaErrorNotSupported;
    } else {
      k_trailq<NC, Prec, MRT><<<(unsigned)A.G, kTQThreads, 0, s>>>(P, (S*)f, st, t_dev, A);
      return cudaGetLastError();
    }
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
    const unsigned nb = std::min<unsigned>(blocks(P), (unsigned)kMassBlocks);  // partial holds blocks(P) rows
    MassShift sh{};
    for (int c = 0; c < NC; ++c) sh.v[c] = (double)P.N * P.rho_ref[c];
    k_mass_partial<Q, NC, Prec><<<nb, kBlock, 0, s>>>(P, (const S*)f, partial);
    k_mass_final<<<1, kBlock, 0, s>>>(partial, (int)nb, NC, sh, out);
  }
  static const Ops* table() {
    static const Ops ops = {psi,           collide,           fused,        fused_max_blocks, fused3,
                            fused3_max_blocks, init,          get_f,        set_f,            fields,
                            mass,          (int)sizeof(S),    (int)sizeof(PsiT), (int)sizeof(R), Fused<Q>::TX,
                            Fused<Q>::TY,  Fused<Q>::P,       kF3WorkersPerCta,  kF3FlagSets,       collide_oop,
                            trail3,        trail3_max_blocks, trailq,     trailq_max_blocks, kTQChunk,
                            kTQLag};
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

}  // namespace lbm
