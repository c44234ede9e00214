// Device-side building blocks of the multi-component pseudo-potential LB step
// (Peng, Ayala & Ayala, arXiv:1909.12390): lattice tables, the MRT moment basis, the
// in-place AA streaming addresses, the mixture Peng-Robinson EOS, the Kupershtokh force
// and the Guo-forced BGK / MRT collision. Everything is a compile-time function of the
// direction index so that fully unrolled loops fold every lattice constant.
#pragma once

#include <cmath>
#include <cstdint>

namespace lbm {

// ---------------------------------------------------------------------------------------
// Lattices. Direction order is part of the ABI (include/lbm.h).
template <int Q>
struct Lat;

template <>
struct Lat<9> {
  static constexpr int D = 2;
  __host__ __device__ static constexpr int e(int a, int d) {
    // (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
    return d == 0 ? (a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0))
         : d == 1 ? (a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0))
                  : 0;
  }
  __host__ __device__ static constexpr int c2(int a) { return e(a, 0) * e(a, 0) + e(a, 1) * e(a, 1); }
  __host__ __device__ static constexpr double w(int a) {
    return c2(a) == 0 ? 4.0 / 9.0 : (c2(a) == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a - 1 + 2) % 4) + 1 : ((a - 5 + 2) % 4) + 5);
  }
  // Lallemand & Luo (2000) moment rows: rho e eps jx qx jy qy pxx pxy
  __host__ __device__ static constexpr int m(int k, int a) {
    return k == 0 ? 1
         : k == 1 ? -4 + 3 * c2(a)
         : k == 2 ? (8 - 21 * c2(a) + 9 * c2(a) * c2(a)) / 2
         : k == 3 ? e(a, 0)
         : k == 4 ? (-5 + 3 * c2(a)) * e(a, 0)
         : k == 5 ? e(a, 1)
         : k == 6 ? (-5 + 3 * c2(a)) * e(a, 1)
         : k == 7 ? e(a, 0) * e(a, 0) - e(a, 1) * e(a, 1)
                  : e(a, 0) * e(a, 1);
  }
  // Rows with a free relaxation rate; rho, j and the stress rows relax at 1/tau.
  static constexpr int NK = 4;
  __host__ __device__ static constexpr int krow(int i) { return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 4 : 6; }
  // pairs of opposite directions: first member of pair p (the other is opp)
  static constexpr int NPAIR = 4;
  __host__ __device__ static constexpr int pfirst(int p) { return p == 0 ? 1 : p == 1 ? 2 : p == 2 ? 5 : 6; }
};

template <>
struct Lat<19> {
  static constexpr int D = 3;
  __host__ __device__ static constexpr int e(int a, int d) {
    // 0:(0,0,0) 1:(1,0,0) 2:(-1,0,0) 3:(0,1,0) 4:(0,-1,0) 5:(0,0,1) 6:(0,0,-1)
    // 7:(1,1,0) 8:(-1,-1,0) 9:(1,-1,0) 10:(-1,1,0) 11:(1,0,1) 12:(-1,0,-1) 13:(1,0,-1)
    // 14:(-1,0,1) 15:(0,1,1) 16:(0,-1,-1) 17:(0,1,-1) 18:(0,-1,1)
    return d == 0 ? (a == 1 || a == 7 || a == 9 || a == 11 || a == 13 ? 1
                     : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14 ? -1 : 0))
         : d == 1 ? (a == 3 || a == 7 || a == 10 || a == 15 || a == 17 ? 1
                     : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18 ? -1 : 0))
                  : (a == 5 || a == 11 || a == 14 || a == 15 || a == 18 ? 1
                     : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17 ? -1 : 0));
  }
  __host__ __device__ static constexpr int c2(int a) {
    return e(a, 0) * e(a, 0) + e(a, 1) * e(a, 1) + e(a, 2) * e(a, 2);
  }
  __host__ __device__ static constexpr double w(int a) {
    return c2(a) == 0 ? 1.0 / 3.0 : (c2(a) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : (a % 2 == 1 ? a + 1 : a - 1); }
  // d'Humieres et al. (2002) moment rows: rho e eps jx qx jy qy jz qz 3pxx 3pixx pww piww
  // pxy pyz pxz mx my mz
  __host__ __device__ static constexpr int m(int k, int a) {
    return k == 0 ? 1
         : k == 1 ? 19 * c2(a) - 30
         : k == 2 ? (21 * c2(a) * c2(a) - 53 * c2(a) + 24) / 2
         : k == 3 ? e(a, 0)
         : k == 4 ? (5 * c2(a) - 9) * e(a, 0)
         : k == 5 ? e(a, 1)
         : k == 6 ? (5 * c2(a) - 9) * e(a, 1)
         : k == 7 ? e(a, 2)
         : k == 8 ? (5 * c2(a) - 9) * e(a, 2)
         : k == 9 ? 3 * e(a, 0) * e(a, 0) - c2(a)
         : k == 10 ? (3 * c2(a) - 5) * (3 * e(a, 0) * e(a, 0) - c2(a))
         : k == 11 ? e(a, 1) * e(a, 1) - e(a, 2) * e(a, 2)
         : k == 12 ? (3 * c2(a) - 5) * (e(a, 1) * e(a, 1) - e(a, 2) * e(a, 2))
         : k == 13 ? e(a, 0) * e(a, 1)
         : k == 14 ? e(a, 1) * e(a, 2)
         : k == 15 ? e(a, 0) * e(a, 2)
         : k == 16 ? (e(a, 1) * e(a, 1) - e(a, 2) * e(a, 2)) * e(a, 0)
         : k == 17 ? (e(a, 2) * e(a, 2) - e(a, 0) * e(a, 0)) * e(a, 1)
                   : (e(a, 0) * e(a, 0) - e(a, 1) * e(a, 1)) * e(a, 2);
  }
  static constexpr int NPAIR = 9;
  __host__ __device__ static constexpr int pfirst(int p) { return 2 * p + 1; }
  static constexpr int NK = 10;
  __host__ __device__ static constexpr int krow(int i) {
    return i == 0 ? 1 : i == 1 ? 2 : i == 2 ? 4 : i == 3 ? 6 : i == 4 ? 8
         : i == 5 ? 10 : i == 6 ? 12 : i == 7 ? 16 : i == 8 ? 17 : 18;
  }
};

template <int Q>
__host__ __device__ constexpr int mnorm(int k) {
  int s = 0;
  for (int a = 0; a < Q; ++a) s += Lat<Q>::m(k, a) * Lat<Q>::m(k, a);
  return s;
}

// Pair structure. The Q - 1 moving directions form NPAIR pairs (a, opp(a)), a = pfirst(p).
// A moment row is even (m(k, opp a) = m(k, a)) or odd (m(k, opp a) = -m(k, a), m(k, 0) = 0):
// row_parity returns +1, -1, or 0 for neither (no row of either basis).
template <int Q>
__host__ __device__ constexpr int row_parity(int k) {
  bool ev = true, od = Lat<Q>::m(k, 0) == 0;
  for (int p = 0; p < Lat<Q>::NPAIR; ++p) {
    const int a = Lat<Q>::pfirst(p), b = Lat<Q>::opp(a);
    ev = ev && Lat<Q>::m(k, b) == Lat<Q>::m(k, a);
    od = od && Lat<Q>::m(k, b) == -Lat<Q>::m(k, a);
  }
  return ev ? 1 : (od ? -1 : 0);
}
// Class of pair p: the axes its directions move along (bit d set when e_d != 0). Entries of the
// even rows with a free rate (energy, energy square, normal-stress-like rows) depend on e_d^2
// only, so they take one value per class (the off-diagonal stress rows e_x e_y do not, and
// relax at 1/tau).
template <int Q>
__host__ __device__ constexpr int pclass(int p) {
  const int a = Lat<Q>::pfirst(p);
  return (Lat<Q>::e(a, 0) != 0 ? 1 : 0) | (Lat<Q>::e(a, 1) != 0 ? 2 : 0) | (Lat<Q>::e(a, 2) != 0 ? 4 : 0);
}
// First pair of class c, or -1.
template <int Q>
__host__ __device__ constexpr int crep(int c) {
  for (int p = 0; p < Lat<Q>::NPAIR; ++p)
    if (pclass<Q>(p) == c) return p;
  return -1;
}
template <int Q>
__host__ __device__ constexpr bool pairs_consistent() {
  int seen = 0;
  for (int p = 0; p < Lat<Q>::NPAIR; ++p) {
    const int a = Lat<Q>::pfirst(p), b = Lat<Q>::opp(a);
    if (a == b || a == 0 || Lat<Q>::opp(b) != a || ((seen >> a) & 1) || ((seen >> b) & 1)) return false;
    seen |= (1 << a) | (1 << b);
    for (int i = 0; i < Lat<Q>::NK; ++i) {  // even free rows: one value per class
      const int k = Lat<Q>::krow(i);
      if (row_parity<Q>(k) == 1 && Lat<Q>::m(k, a) != Lat<Q>::m(k, Lat<Q>::pfirst(crep<Q>(pclass<Q>(p)))))
        return false;
    }
  }
  for (int k = 0; k < Q; ++k)
    if (row_parity<Q>(k) == 0) return false;
  return seen == (1 << Q) - 2;
}
static_assert(pairs_consistent<9>() && pairs_consistent<19>(), "lattice pair tables");

// ---------------------------------------------------------------------------------------
// Parameters of one lattice, passed by value to every kernel.
struct Params {
  int nx, ny, nz;
  int64_t N;  // nx * ny * nz
  uint32_t N32;
  int nc;
  // collision
  double omega;      // 1 / tau
  double lam[10];    // (s_k - 1/tau) / |row k|^2 for the free MRT rows, in Lat<Q>::krow order
  // EOS, Section 3.2 (FP64)
  double invM[4];    // 1 / M_i
  double b[4];       // b_i (molar co-volume)
  double Qa[16];     // sqrt(a_i alpha_i a_j alpha_j) (1 - zeta_ij)
  double sa[4];      // sqrt(a_i alpha_i)
  int kij_zero;      // every zeta_ij == 0: [a alpha]_m n^2 = (sum_i n_i sa_i)^2
  float invMf[4];    // 1 / M_i in FP32
  double RT;
  double cpsi;       // 2 / (G cs2): psi^2 = cpsi (p - cs2 rho)
  double rho_ref[4]; // FP32 shift references (0 for FP64 storage)
  double gamma[4];
  double beta, G;
  int split;          // LBM_SPLIT_VOLATILITY (0) or LBM_SPLIT_GONG (1)
  // constants derived by finalize_params(), in both precisions, so that no kernel converts a
  // parameter per site (an FP64 -> FP32 conversion runs on GB300's 1/72-rate FP64 pipe)
  double gk, c1, c2;  // 1 - omega/2, -beta G, -(1 - beta) G / 2
  double k1, k2;      // pair form of the force: -G / 36, -(1 - beta) G / 72 (weights counted in 1/36)
  float omega_f, gk_f, c1_f, c2_f, cpsi_f, k1_f, k2_f;
  float lam_f[10], rho_ref_f[4], gamma_f[4];
  // the FP32-input EOS works with p / RT: sa_i / sqrt(RT), Qa_ii / RT and 2 Qa_ij / RT (i < j);
  // psi^2 = cpsi RT (p / RT - rho / (3 RT))
  double sa_rt[4], Qa_rt[16];
  float cpsi_rt_f, c3rt_f;
  // FP32 copies for the adjoint of FP32-shifted storage
  float b_f[4], Qa_f[16], sa_f[4], RT_f;
};

// Fills the derived constants of P (call after any change of omega, lam, rho_ref, gamma,
// beta, G or cpsi).
inline void finalize_params(Params& P) {
  P.gk = 1.0 - 0.5 * P.omega;
  P.c1 = -P.beta * P.G;
  P.c2 = -0.5 * (1.0 - P.beta) * P.G;
  P.k1 = -P.G / 36.0;
  P.k2 = -0.5 * (1.0 - P.beta) * P.G / 36.0;
  P.k1_f = (float)P.k1;
  P.k2_f = (float)P.k2;
  P.omega_f = (float)P.omega;
  P.gk_f = (float)P.gk;
  P.c1_f = (float)P.c1;
  P.c2_f = (float)P.c2;
  P.cpsi_f = (float)P.cpsi;
  for (int i = 0; i < 10; ++i) P.lam_f[i] = (float)P.lam[i];
  for (int i = 0; i < 4; ++i) {
    P.rho_ref_f[i] = (float)P.rho_ref[i];
    P.gamma_f[i] = (float)P.gamma[i];
  }
  for (int i = 0; i < 4; ++i) {
    P.sa_rt[i] = P.RT > 0 ? P.sa[i] / std::sqrt(P.RT) : 0.0;
    for (int j = 0; j < 4; ++j) P.Qa_rt[i * 4 + j] = P.RT > 0 ? (i == j ? 1.0 : 2.0) * P.Qa[i * 4 + j] / P.RT : 0.0;
  }
  for (int i = 0; i < 4; ++i) {
    P.b_f[i] = (float)P.b[i];
    P.sa_f[i] = (float)P.sa[i];
  }
  for (int i = 0; i < 16; ++i) P.Qa_f[i] = (float)P.Qa[i];
  P.RT_f = (float)P.RT;
  P.cpsi_rt_f = (float)(P.cpsi * P.RT);
  P.c3rt_f = P.RT > 0 ? (float)(1.0 / (3.0 * P.RT)) : 0.0f;
}

// Per-site constants in the arithmetic precision R of a kernel.
template <class R>
struct PC;
template <>
struct PC<double> {
  __device__ __forceinline__ static double omega(const Params& P) { return P.omega; }
  __device__ __forceinline__ static double gk(const Params& P) { return P.gk; }
  __device__ __forceinline__ static double c1(const Params& P) { return P.c1; }
  __device__ __forceinline__ static double c2(const Params& P) { return P.c2; }
  __device__ __forceinline__ static double k1(const Params& P) { return P.k1; }
  __device__ __forceinline__ static double k2(const Params& P) { return P.k2; }
  __device__ __forceinline__ static double lam(const Params& P, int i) { return P.lam[i]; }
  __device__ __forceinline__ static double rho_ref(const Params& P, int i) { return P.rho_ref[i]; }
  __device__ __forceinline__ static double gamma(const Params& P, int i) { return P.gamma[i]; }
  __device__ __forceinline__ static double invM(const Params& P, int i) { return P.invM[i]; }
  __device__ __forceinline__ static double cpsi(const Params& P) { return P.cpsi; }
};
template <>
struct PC<float> {
  __device__ __forceinline__ static float omega(const Params& P) { return P.omega_f; }
  __device__ __forceinline__ static float gk(const Params& P) { return P.gk_f; }
  __device__ __forceinline__ static float c1(const Params& P) { return P.c1_f; }
  __device__ __forceinline__ static float c2(const Params& P) { return P.c2_f; }
  __device__ __forceinline__ static float k1(const Params& P) { return P.k1_f; }
  __device__ __forceinline__ static float k2(const Params& P) { return P.k2_f; }
  __device__ __forceinline__ static float lam(const Params& P, int i) { return P.lam_f[i]; }
  __device__ __forceinline__ static float rho_ref(const Params& P, int i) { return P.rho_ref_f[i]; }
  __device__ __forceinline__ static float gamma(const Params& P, int i) { return P.gamma_f[i]; }
  __device__ __forceinline__ static float invM(const Params& P, int i) { return P.invMf[i]; }
  __device__ __forceinline__ static float cpsi(const Params& P) { return P.cpsi_f; }
};

// Status bits raised by kernels (OR-ed into one device word).
enum : int { ST_PSI_DOMAIN = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4 };

// ---------------------------------------------------------------------------------------
// Site coordinates and periodic neighbours. Site indices are 32-bit: the host requires
// Q * N < 2^32 (offsets inside one component's block of Q * N populations).
struct Site {
  uint32_t idx;
  int x, y, z;
  int xm, xp, ym, yp, zm, zp;
  __device__ __forceinline__ void set_xyz(const Params& P, int x_, int y_, int z_) {
    x = x_;
    y = y_;
    z = z_;
    idx = ((uint32_t)z * (uint32_t)P.ny + (uint32_t)y) * (uint32_t)P.nx + (uint32_t)x;
    xm = x == 0 ? P.nx - 1 : x - 1;
    xp = x == P.nx - 1 ? 0 : x + 1;
    ym = y == 0 ? P.ny - 1 : y - 1;
    yp = y == P.ny - 1 ? 0 : y + 1;
    zm = z == 0 ? P.nz - 1 : z - 1;
    zp = z == P.nz - 1 ? 0 : z + 1;
  }
  __device__ __forceinline__ void set(const Params& P, uint32_t i) {
    const uint32_t r = i / (uint32_t)P.nx;
    set_xyz(P, (int)(i - r * (uint32_t)P.nx), (int)(r % (uint32_t)P.ny), (int)(r / (uint32_t)P.ny));
  }
  // linear index of the site x + (ex, ey, ez), each component in {-1, 0, 1}
  __device__ __forceinline__ uint32_t nb(const Params& P, int ex, int ey, int ez) const {
    const int xx = ex == 0 ? x : (ex > 0 ? xp : xm);
    const int yy = ey == 0 ? y : (ey > 0 ? yp : ym);
    const int zz = ez == 0 ? z : (ez > 0 ? zp : zm);
    return ((uint32_t)zz * (uint32_t)P.ny + (uint32_t)yy) * (uint32_t)P.nx + (uint32_t)xx;
  }
};

// In-place AA streaming. State at even t: slot (x, a) holds f_a(x, t). After an even step
// slot (x, opp a) holds f*_a(x) = f_a(x + e_a, t + 1), so at odd t f_a(x) sits in slot
// (x - e_a, opp a); the odd step writes f*_a(x) to slot (x + e_a, a), which restores the even
// layout. Each site reads and writes the same slots, so no two threads touch one slot.
// Offsets are relative to the start of one component's block of Q * N values; PAR is the
// parity of the step (a template argument, so each kernel is compiled once per parity).
template <int Q>
struct AA {
  template <int A, int PAR>
  __device__ __forceinline__ static uint32_t rd(const Params& P, const Site& s) {
    constexpr int O = Lat<Q>::opp(A);
    if constexpr (PAR == 0) return (uint32_t)A * P.N32 + s.idx;
    return (uint32_t)O * P.N32 + s.nb(P, -Lat<Q>::e(A, 0), -Lat<Q>::e(A, 1), -Lat<Q>::e(A, 2));
  }
  template <int A, int PAR>
  __device__ __forceinline__ static uint32_t wr(const Params& P, const Site& s) {
    constexpr int O = Lat<Q>::opp(A);
    if constexpr (PAR == 0) return (uint32_t)O * P.N32 + s.idx;
    return (uint32_t)A * P.N32 + s.nb(P, Lat<Q>::e(A, 0), Lat<Q>::e(A, 1), Lat<Q>::e(A, 2));
  }
};

// Start of component c's block of Q * N populations.
template <int Q, class T>
__device__ __forceinline__ T* comp_base(T* f, const Params& P, int c) {
  return f + (size_t)c * Q * P.N;
}

// Multiply-add with one rounding. The library is compiled with -fmad=false, so the compiler
// forms no multiply-add of its own: every one is written out here, and the per-site code
// rounds identically in every kernel that inlines it (the paths are compared bit for bit).
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

// Compile-time loop.
template <int I, int N>
struct For {
  template <class F>
  __device__ __forceinline__ static void run(F&& f) {
    f.template operator()<I>();
    For<I + 1, N>::run(f);
  }
};
template <int N>
struct For<N, N> {
  template <class F>
  __device__ __forceinline__ static void run(F&&) {}
};

// ---------------------------------------------------------------------------------------
// Mixture Peng-Robinson EOS (Eq. MCPengRobinson with Eq. randommixingrule), written without
// the division by the molar density: with n_i = rho_i / M_i, n = sum n_i,
//   b_m n = sum b_i n_i = B,   [a alpha]_m n^2 = sum_ij n_i n_j Qa_ij = A2,
//   p = n R T / (1 - B) - A2 / (1 + 2B - B^2).
// Returns the numerator pD = n R T (1 + 2B - B^2) - A2 (1 - B) and the denominator
// Dd = (1 - B)(1 + 2B - B^2), both FP64, so p = pD / Dd. Every sum with cancellation is FP64.
template <int NC>
struct EosOut {
  double pD, Dd, B;
};

template <int NC>
__device__ __forceinline__ EosOut<NC> eos_pr(const Params& P, const double (&rho)[NC]) {
  double n[NC];
  double nt = 0.0, B = 0.0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    n[i] = rho[i] * P.invM[i];
    nt += n[i];
    B = fma(P.b[i], n[i], B);
  }
  double A2 = 0.0;
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    double v = P.Qa[i * 4 + i] * n[i];
#pragma unroll
    for (int j = i + 1; j < NC; ++j) v = fma(2.0 * P.Qa[i * 4 + j], n[j], v);
    A2 = fma(n[i], v, A2);
  }
  double d1 = 1.0 - B;
  double d2 = fma(B, 2.0 - B, 1.0);
  EosOut<NC> o;
  o.Dd = d1 * d2;
  o.pD = fma(nt * P.RT, d2, -A2 * d1);
  o.B = B;
  return o;
}

// Conversions between binary32 and binary64 in integer arithmetic (IEEE 754 formats). On
// GB300 a conversion instruction occupies the FP64 pipe like an FP64 multiply-add, and the
// pseudo-potential pass is bound by that pipe; the integer forms below run on the integer
// pipes. Each covers the common case exactly and reports whether it applies; callers fall back
// to the conversion instruction, warp by warp, for the rest.
//
// Widening of a normal binary32 value (exact): the sign carries over, the biased exponent
// gains 1023 - 127 = 896 and the 23 fraction bits become the top 23 of the 52.
__device__ __forceinline__ bool widen_int_ok(float x) {
  return (__float_as_uint(x) & 0x7fffffffu) - 0x00800000u < 0x7f000000u;  // biased exponent 1 .. 254
}
__device__ __forceinline__ double widen_int(float x) {
  const unsigned u = __float_as_uint(x), m = u & 0x7fffffffu;
  return __hiloint2double((int)(((m >> 3) + 0x38000000u) | (u & 0x80000000u)), (int)(u << 29));
}
// Narrowing with round to nearest, ties to even, for |x| whose binary32 result is a normal
// number or overflows to infinity: biased binary64 exponent 897 .. 1150. The 23 fraction bits
// are the top of the 52, the 29 bits below them decide the rounding, and a carry out of the
// fraction increments the exponent (up to infinity), as rounding requires.
__device__ __forceinline__ bool narrow_int_ok(double x) {
  return ((unsigned)__double2hiint(x) & 0x7fffffffu) - 0x38100000u < 0x0fe00000u;
}
__device__ __forceinline__ float narrow_int(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  unsigned f = (((hi & 0x7fffffffu) - 0x38000000u) << 3) | (lo >> 29);
  const unsigned r = lo & 0x1fffffffu;
  f += (unsigned)(r > 0x10000000u) | ((unsigned)(r == 0x10000000u) & (f & 1u));
  return __uint_as_float(f | (hi & 0x80000000u));
}
// Element-wise conversions of small arrays; a warp takes the conversion instruction only when
// one of its lanes has a value outside the integer forms' range.
template <int N>
__device__ __forceinline__ void widen_all(const float (&x)[N], double (&y)[N]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y[i] = widen_int(x[i]);
    ok = ok && widen_int_ok(x[i]);
  }
  if (__any_sync(__activemask(), !ok)) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (!widen_int_ok(x[i])) y[i] = (double)x[i];
  }
}
template <int N>
__device__ __forceinline__ void narrow_all(const double (&x)[N], float (&y)[N]) {
  bool ok = true;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    y[i] = narrow_int(x[i]);
    ok = ok && narrow_int_ok(x[i]);
  }
  if (__any_sync(__activemask(), !ok)) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (!narrow_int_ok(x[i])) y[i] = (float)x[i];
  }
}

// The same pressure from FP32 cell-volume densities (FP32-shifted storage), returned as
// pD / Dd = p / RT. The molar densities n_i = rho_i / M_i are formed in FP32 (their inputs
// carry FP32 precision) and widened exactly; every sum of the EOS and the numerator with its
// cancellation run in FP64:
//   B = sum b_i n_i,  A2' = sum_ij n_i n_j Qa_ij / RT  (= (sum_i n_i sa_i / sqrt(RT))^2 when
//   all zeta_ij = 0),  d1 = 1 - B,  d2 = 1 + 2B - B^2 = 2 - d1^2,
//   pD = n d2 - A2' d1,  Dd = d1 d2.
// Dividing through by RT saves the multiplication n RT; d2 from d1 saves the subtraction 2 - B.
// ok is B < 1 (d1 > 0), tested on the sign and exponent bits of d1.
struct EosOutF {
  double pD, Dd;
  bool ok;
};

template <int NC>
__device__ __forceinline__ EosOutF eos_pr_f32in(const Params& P, const float (&rho)[NC]) {
  float nf[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) nf[i] = rho[i] * P.invMf[i];
  double n[NC];
  widen_all<NC>(nf, n);
  double nt = n[0], B = P.b[0] * n[0];
#pragma unroll
  for (int i = 1; i < NC; ++i) {
    nt += n[i];
    B = fma(P.b[i], n[i], B);
  }
  double A2;
  if (P.kij_zero) {
    double S = P.sa_rt[0] * n[0];
#pragma unroll
    for (int i = 1; i < NC; ++i) S = fma(P.sa_rt[i], n[i], S);
    A2 = S * S;
  } else {
    A2 = 0.0;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      double v = P.Qa_rt[i * 4 + i] * n[i];
#pragma unroll
      for (int j = i + 1; j < NC; ++j) v = fma(P.Qa_rt[i * 4 + j], n[j], v);
      A2 = fma(n[i], v, A2);
    }
  }
  const double d1 = 1.0 - B;
  const double d2 = fma(-d1, d1, 2.0);
  EosOutF o;
  o.Dd = d1 * d2;
  o.pD = fma(nt, d2, -A2 * d1);
  o.ok = __double2hiint(d1) > 0;
  return o;
}

}  // namespace lbm
