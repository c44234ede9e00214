// FP64 CPU oracle of the time step of the thermodynamically consistent multi-component
// pseudo-potential lattice Boltzmann model of Peng, Ayala & Ayala (arXiv:1909.12390).
//
// TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
// reference leg may load or call this file. It shares no code with the CUDA library and the
// CUDA library never calls it.
//
// It is deliberately plain: double-buffered populations, three whole-grid loops per step
// (moments + EOS + pseudo-potential into arrays, then force + split + collision into a
// post-collision buffer, then a periodic shift for streaming), no fusion, no reordering
// beyond what the equations state. It is templated on the scalar type so that a two-direction
// dual number gives forward-mode derivatives with respect to the binary interaction
// coefficients and the volatility coefficients.
//
// Step order follows Section 3.4 (implementation list):
//   1. cell-volume densities  rho_s = sum_a f_{s,a}                            (Eq. LBE context)
//   2. mixture Peng-Robinson pressure at the local molar density and molar
//      composition                                       (Eq. MCPengRobinson, Eq. randommixingrule)
//   3. pseudo-potential psi = sqrt(2 (p_EOS - cs2 rho) / (G cs2))             (Eq. psicorrected)
//   4. total force, Kupershtokh beta form                                     (Eq. coupledMCforce)
//   5. split  F_s = chi_s F,  chi_s = gamma_s rho_s / sum_j gamma_j rho_j      (Eq. distributionforce)
//   6. BGK collision with Guo forcing per component             (Eq. LBE, Eq. equilibrium a, b)
//      or its multiple-relaxation-time analogue (not in the paper)
//   7. streaming f(x + e_a, t + 1) = f*(x, t) on a periodic grid              (Eq. LBE)
//
// Readings of points the paper leaves open (lattice units dt = dx = 1, cs2 = 1/3):
//   * lattice: D2Q9 for 2-D, D3Q19 for 3-D, standard weights; the force stencil uses the
//     lattice weights w_a.
//   * the shared velocity of Eq. equilibrium is the barycentric one with the Guo half force:
//     rho u = sum_s sum_a e_a f_{s,a} + F / 2, rho = sum_s rho_s, F = sum_s F_s.
//   * the EOS is evaluated at the molar density n = sum_i rho_i / M_i with the molar
//     composition c_i = (rho_i / M_i) / n; the cs2 rho term of Eq. psicorrected uses the mass
//     density rho = sum_i rho_i.
//   * a_i, b_i, alpha_i, m_i as in Section 3.2 with Omega_a = 0.45724, Omega_b = 0.0778.
//   * psi^2 < 0 is a domain error; nothing is clamped.
//   * MRT (not in the paper): m = M f, m* = m - S (m - M f_eq) + (I - S/2) M Fbar, f* = M^-1 m*,
//     Fbar the Guo term without its (1 - 1/2tau) factor, M^-1 by Gauss-Jordan elimination.
#include <omp.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

namespace {

const double CS2 = 1.0 / 3.0;
const double OMEGA_A = 0.45724;
const double OMEGA_B = 0.0778;

// ---- scalar types --------------------------------------------------------------------------
struct Dual {  // value and derivatives along two directions
  double v, d0, d1;
  Dual() : v(0), d0(0), d1(0) {}
  Dual(double a) : v(a), d0(0), d1(0) {}
  Dual(double a, double b, double c) : v(a), d0(b), d1(c) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d0 + b.d0, a.d1 + b.d1); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d0 - b.d0, a.d1 - b.d1); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d0, -a.d1); }
inline Dual operator*(Dual a, Dual b) {
  return Dual(a.v * b.v, a.d0 * b.v + a.v * b.d0, a.d1 * b.v + a.v * b.d1);
}
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d0 - q * b.d0) / b.v, (a.d1 - q * b.d1) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual sqrt_(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, a.d0 / (2 * s), a.d1 / (2 * s));
}
inline double sqrt_(double a) { return std::sqrt(a); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }

// ---- lattices ------------------------------------------------------------------------------
struct Lattice {
  int D, Q;
  int e[19][3];
  double w[19];
};

Lattice make_lattice(int Q) {
  Lattice L;
  std::memset(&L, 0, sizeof(L));
  L.Q = Q;
  if (Q == 9) {
    L.D = 2;
    const int E[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                         {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int a = 0; a < 9; ++a) {
      L.e[a][0] = E[a][0];
      L.e[a][1] = E[a][1];
      L.e[a][2] = 0;
      int c2 = E[a][0] * E[a][0] + E[a][1] * E[a][1];
      L.w[a] = c2 == 0 ? 4.0 / 9.0 : (c2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
  } else {
    L.D = 3;
    const int E[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                          {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                          {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                          {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    for (int a = 0; a < 19; ++a) {
      int c2 = 0;
      for (int d = 0; d < 3; ++d) {
        L.e[a][d] = E[a][d];
        c2 += E[a][d] * E[a][d];
      }
      L.w[a] = c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
  }
  return L;
}

// Moment basis of the MRT collision, one polynomial in the velocity components per row:
// D2Q9 after Lallemand & Luo (2000), D3Q19 after d'Humieres et al. (2002).
double moment_row(int Q, int k, const int* e) {
  double x = e[0], y = e[1], z = e[2];
  double c2 = x * x + y * y + z * z;
  if (Q == 9) {
    switch (k) {
      case 0: return 1;
      case 1: return -4 + 3 * c2;
      case 2: return 4 - 10.5 * c2 + 4.5 * c2 * c2;
      case 3: return x;
      case 4: return (-5 + 3 * c2) * x;
      case 5: return y;
      case 6: return (-5 + 3 * c2) * y;
      case 7: return x * x - y * y;
      default: return x * y;
    }
  }
  switch (k) {
    case 0: return 1;
    case 1: return 19 * c2 - 30;
    case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * c2 - 9) * x;
    case 5: return y;
    case 6: return (5 * c2 - 9) * y;
    case 7: return z;
    case 8: return (5 * c2 - 9) * z;
    case 9: return 3 * x * x - c2;
    case 10: return (3 * c2 - 5) * (3 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3 * c2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
  }
}

// Gauss-Jordan inverse with partial pivoting, n <= 19. Returns false if singular.
bool invert(int n, const double* A, double* Ainv) {
  double a[19][38];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      a[i][j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[p][c])) p = r;
    if (std::fabs(a[p][c]) < 1e-14) return false;
    if (p != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(a[p][j], a[c][j]);
    double piv = a[c][c];
    for (int j = 0; j < 2 * n; ++j) a[c][j] /= piv;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double m = a[r][c];
      if (m == 0) continue;
      for (int j = 0; j < 2 * n; ++j) a[r][j] -= m * a[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = a[i][j + n];
  return true;
}

}  // namespace

extern "C" {

// Problem description; every quantity in lattice units (R = gas constant, normally 1).
typedef struct {
  int Q;           // 9 (D2Q9) or 19 (D3Q19)
  int nx, ny, nz;  // nz = 1 for D2Q9
  int nc;          // number of components, 1..4
  double tau;      // BGK relaxation time (Eq. LBE)
  int collision;   // 0 = BGK, 1 = MRT
  double s[19];    // MRT relaxation rate of each moment row (collision == 1)
  double T, R;     // temperature and gas constant
  double Tc[4], pc[4], omega[4], M[4];  // critical constants and molar masses
  double kij[16];  // binary interaction coefficients zeta_ij, row-major nc x nc
  double gamma[4]; // volatility coefficients gamma_i of Eq. distributionforce
  double beta, G;  // Kupershtokh beta and interaction strength (Eq. coupledMCforce)
  int split;       // 0: Eq. distributionforce (gamma); 1: Eq. Gong, |p0 - ph_i| (FP64 only)
} oracle_case;

enum { ORACLE_OK = 0, ORACLE_ERR_ARG = -1, ORACLE_ERR_PSI_DOMAIN = -4, ORACLE_ERR_NONFINITE = -5 };

}  // extern "C"

namespace {

struct Setup {
  Lattice L;
  int nx, ny, nz, nc;
  int64_t N;
  double tau;
  int collision;
  double s[19];
  double Mm[19 * 19], Minv[19 * 19];
  double RT, G, beta;
  double aalpha[4], b[4], M[4];
  int split;
};

// a_i, b_i, alpha_i(T), m_i of Section 3.2 (Eq. SCpengrobinson's mixture counterpart).
void component_parameters(const oracle_case* c, Setup* S) {
  for (int i = 0; i < c->nc; ++i) {
    double w = c->omega[i];
    double m = w <= 0.49 ? 0.374640 + 1.54226 * w - 0.26992 * w * w
                         : 0.379642 + 1.48503 * w - 0.164423 * w * w + 0.016666 * w * w * w;
    double a = OMEGA_A * c->R * c->R * c->Tc[i] * c->Tc[i] / c->pc[i];
    double bb = OMEGA_B * c->R * c->Tc[i] / c->pc[i];
    double sq = 1 + m * (1 - std::sqrt(c->T / c->Tc[i]));
    S->aalpha[i] = a * sq * sq;
    S->b[i] = bb;
    S->M[i] = c->M[i];
  }
}

int make_setup(const oracle_case* c, Setup* S) {
  if (!c || (c->Q != 9 && c->Q != 19) || c->nc < 1 || c->nc > 4 || c->nx < 1 || c->ny < 1 ||
      c->nz < 1 || (c->Q == 9 && c->nz != 1) || !(c->tau > 0.5))
    return ORACLE_ERR_ARG;
  S->L = make_lattice(c->Q);
  S->nx = c->nx; S->ny = c->ny; S->nz = c->nz; S->nc = c->nc;
  S->N = (int64_t)c->nx * c->ny * c->nz;
  S->tau = c->tau;
  S->collision = c->collision;
  if (c->split != 0 && c->split != 1) return ORACLE_ERR_ARG;
  S->split = c->split;
  for (int k = 0; k < 19; ++k) S->s[k] = c->s[k];
  S->RT = c->R * c->T;
  S->G = c->G;
  S->beta = c->beta;
  component_parameters(c, S);
  if (c->collision == 1) {
    int Q = c->Q;
    for (int k = 0; k < Q; ++k)
      for (int a = 0; a < Q; ++a) S->Mm[k * Q + a] = moment_row(Q, k, S->L.e[a]);
    if (!invert(Q, S->Mm, S->Minv)) return ORACLE_ERR_ARG;
  }
  return ORACLE_OK;
}

inline int64_t site(const Setup& S, int x, int y, int z) {
  return ((int64_t)z * S.ny + y) * S.nx + x;
}
inline int64_t neighbour(const Setup& S, int x, int y, int z, const int* e) {
  int xx = ((x + e[0]) % S.nx + S.nx) % S.nx;
  int yy = ((y + e[1]) % S.ny + S.ny) % S.ny;
  int zz = ((z + e[2]) % S.nz + S.nz) % S.nz;
  return site(S, xx, yy, zz);
}

// Mixture Peng-Robinson pressure (Eq. MCPengRobinson) with the random mixing rules
// (Eq. randommixingrule), evaluated at the molar density and molar composition of the
// cell-volume densities rho_c; then psi^2 of Eq. psicorrected.
template <class T>
int eos(const Setup& S, const T* kij, const T* rho_c, T* p_out, T* psi2_out) {
  const int nc = S.nc;
  T n[4], c[4];
  T ntot = 0.0;
  for (int i = 0; i < nc; ++i) {
    n[i] = rho_c[i] / T(S.M[i]);
    ntot += n[i];
  }
  if (!(val(ntot) > 0) || !std::isfinite(val(ntot))) return ORACLE_ERR_NONFINITE;
  for (int i = 0; i < nc; ++i) c[i] = n[i] / ntot;
  T aam = 0.0, bm = 0.0;
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j)
      aam += c[i] * c[j] * T(std::sqrt(S.aalpha[i] * S.aalpha[j])) * (T(1.0) - kij[i * nc + j]);
  for (int i = 0; i < nc; ++i) bm += c[i] * T(S.b[i]);
  T p = ntot * T(S.RT) / (T(1.0) - bm * ntot) -
        aam * ntot * ntot / (T(1.0) + T(2.0) * bm * ntot - bm * bm * ntot * ntot);
  T rho = 0.0;
  for (int i = 0; i < nc; ++i) rho += rho_c[i];
  T psi2 = T(2.0) * (p - T(CS2) * rho) / (T(S.G) * T(CS2));
  *p_out = p;
  *psi2_out = psi2;
  if (!std::isfinite(val(psi2))) return ORACLE_ERR_NONFINITE;
  if (val(psi2) < 0) return ORACLE_ERR_PSI_DOMAIN;
  return ORACLE_OK;
}

// Per-site macroscopic state at time t, whole-grid arrays.
template <class T>
struct Macro {
  std::vector<T> rho_c;  // [nc][N] cell-volume densities
  std::vector<T> mom;    // [3][N] sum_s sum_a e_a f
  std::vector<T> p, psi2, psi;  // [N]
  std::vector<T> F;      // [3][N] total force
};

template <class T>
int macroscopic(const Setup& S, const T* kij, const T* f, Macro<T>& m) {
  const int Q = S.L.Q, nc = S.nc;
  const int64_t N = S.N;
  m.rho_c.assign(nc * N, T(0.0));
  m.mom.assign(3 * N, T(0.0));
  m.p.assign(N, T(0.0));
  m.psi2.assign(N, T(0.0));
  m.psi.assign(N, T(0.0));
  m.F.assign(3 * N, T(0.0));
  std::vector<int> site_status(N, ORACLE_OK);
  // Loop 1: moments, EOS, pseudo-potential.
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; ++x) {
    T rc[4];
    for (int s = 0; s < nc; ++s) {
      T acc = 0.0;
      for (int a = 0; a < Q; ++a) {
        T fa = f[((int64_t)s * Q + a) * N + x];
        acc += fa;
        for (int d = 0; d < 3; ++d)
          if (S.L.e[a][d]) m.mom[d * N + x] += T((double)S.L.e[a][d]) * fa;
      }
      rc[s] = acc;
      m.rho_c[s * N + x] = acc;
    }
    T p, psi2;
    int st = eos(S, kij, rc, &p, &psi2);
    if (st != ORACLE_OK) {
      site_status[x] = st;
      continue;
    }
    m.p[x] = p;
    m.psi2[x] = psi2;
    m.psi[x] = sqrt_(psi2);
  }
  for (int64_t x = 0; x < N; ++x)
    if (site_status[x] != ORACLE_OK) return site_status[x];
  // Total force, Eq. coupledMCforce:
  //   F = -beta G psi(x) sum_a w_a psi(x+e_a) e_a - (1 - beta)/2 G sum_a w_a psi^2(x+e_a) e_a
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < S.nz; ++z)
    for (int y = 0; y < S.ny; ++y)
      for (int x = 0; x < S.nx; ++x) {
        int64_t i = site(S, x, y, z);
        T s1[3] = {0.0, 0.0, 0.0}, s2[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < Q; ++a) {
          int64_t j = neighbour(S, x, y, z, S.L.e[a]);
          for (int d = 0; d < 3; ++d) {
            if (!S.L.e[a][d]) continue;
            T ed = T((double)S.L.e[a][d]);
            s1[d] += T(S.L.w[a]) * m.psi[j] * ed;
            s2[d] += T(S.L.w[a]) * m.psi2[j] * ed;
          }
        }
        for (int d = 0; d < 3; ++d)
          m.F[d * N + i] = T(-S.beta * S.G) * m.psi[i] * s1[d] -
                           T(0.5 * (1.0 - S.beta) * S.G) * s2[d];
      }
  return ORACLE_OK;
}

template <class T>
int step_once(const Setup& S, const T* kij, const T* gamma, const T* fin, T* fout) {
  const int Q = S.L.Q, nc = S.nc, D = S.L.D;
  const int64_t N = S.N;
  Macro<T> m;
  int st = macroscopic(S, kij, fin, m);
  if (st != ORACLE_OK) return st;
  std::vector<T> post((size_t)nc * Q * N);
  const double tau = S.tau;
  // Loop 2: split, velocity, collision.
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < N; ++x) {
    T rho = 0.0, gsum = 0.0;
    for (int s = 0; s < nc; ++s) {
      rho += m.rho_c[s * N + x];
      gsum += gamma[s] * m.rho_c[s * N + x];
    }
    T Fx[3], u[3];
    for (int d = 0; d < 3; ++d) {
      Fx[d] = m.F[d * N + x];
      u[d] = (m.mom[d * N + x] + T(0.5) * Fx[d]) / rho;
    }
    T uu = 0.0;
    for (int d = 0; d < D; ++d) uu += u[d] * u[d];
    // Gong et al.'s split (Eq. Gong) with the two pressures under the root put in the order
    // that makes the difference non-negative, as the paper does to keep it real (Section
    // 4.2): chi_i = c_i sqrt(|p0 - ph_i|) / sum_j (...), c_i the molar composition, ph_i the
    // PR pressure of pure i at the mixture's molar density n, p0 = n R T.
    double gong[4] = {0, 0, 0, 0};
    if (S.split == 1) {
      if constexpr (std::is_same_v<T, double>) {
        double nmol[4], nt = 0.0, wsum = 0.0;
        for (int s = 0; s < nc; ++s) {
          nmol[s] = m.rho_c[s * N + x] / S.M[s];
          nt += nmol[s];
        }
        const double p0 = nt * S.RT;
        for (int s = 0; s < nc; ++s) {
          const double b = S.b[s], ph = p0 / (1.0 - b * nt) - S.aalpha[s] * nt * nt / (1.0 + 2.0 * b * nt - b * b * nt * nt);
          gong[s] = nmol[s] / nt * std::sqrt(std::fabs(p0 - ph));
          wsum += gong[s];
        }
        for (int s = 0; s < nc; ++s) gong[s] /= wsum;
      }
    }
    for (int s = 0; s < nc; ++s) {
      T rs = m.rho_c[s * N + x];
      T chi = S.split == 1 ? T(gong[s]) : gamma[s] * rs / gsum;  // Eq. Gong / Eq. distributionforce
      T Fs[3] = {chi * Fx[0], chi * Fx[1], chi * Fx[2]};
      T feq[19], fbar[19], fa[19];
      for (int a = 0; a < Q; ++a) {
        T eu = 0.0, eF = 0.0, uF = 0.0;
        for (int d = 0; d < D; ++d) {
          T ed = T((double)S.L.e[a][d]);
          eu += ed * u[d];
          eF += ed * Fs[d];
          uF += u[d] * Fs[d];
        }
        feq[a] = rs * T(S.L.w[a]) *
                 (T(1.0) + eu / T(CS2) + eu * eu / T(2 * CS2 * CS2) - uu / T(2 * CS2));
        // Guo term without the (1 - 1/2tau) factor: w [(e - u)/cs2 + (e.u) e / cs4] . F_s
        fbar[a] = T(S.L.w[a]) * ((eF - uF) / T(CS2) + eu * eF / T(CS2 * CS2));
        fa[a] = fin[((int64_t)s * Q + a) * N + x];
      }
      if (S.collision == 0) {
        for (int a = 0; a < Q; ++a)
          post[((int64_t)s * Q + a) * N + x] =
              fa[a] - (fa[a] - feq[a]) / T(tau) + T(1.0 - 0.5 / tau) * fbar[a];
      } else {
        T mo[19], meq[19], mf[19], ms[19];
        for (int k = 0; k < Q; ++k) {
          mo[k] = 0.0; meq[k] = 0.0; mf[k] = 0.0;
          for (int a = 0; a < Q; ++a) {
            T Mka = T(S.Mm[k * Q + a]);
            mo[k] += Mka * fa[a];
            meq[k] += Mka * feq[a];
            mf[k] += Mka * fbar[a];
          }
          ms[k] = mo[k] - T(S.s[k]) * (mo[k] - meq[k]) + T(1.0 - 0.5 * S.s[k]) * mf[k];
        }
        for (int a = 0; a < Q; ++a) {
          T acc = 0.0;
          for (int k = 0; k < Q; ++k) acc += T(S.Minv[a * Q + k]) * ms[k];
          post[((int64_t)s * Q + a) * N + x] = acc;
        }
      }
    }
  }
  // Loop 3: periodic streaming.
#pragma omp parallel for collapse(3) schedule(static)
  for (int s = 0; s < nc; ++s)
    for (int a = 0; a < Q; ++a)
      for (int z = 0; z < S.nz; ++z)
        for (int y = 0; y < S.ny; ++y)
          for (int x = 0; x < S.nx; ++x) {
            int64_t i = site(S, x, y, z);
            int64_t j = neighbour(S, x, y, z, S.L.e[a]);
            fout[((int64_t)s * Q + a) * N + j] = post[((int64_t)s * Q + a) * N + i];
          }
  int bad = 0;
#pragma omp parallel for reduction(| : bad) schedule(static)
  for (int64_t k = 0; k < (int64_t)nc * Q * N; ++k)
    if (!std::isfinite(val(fout[k]))) bad = 1;
  return bad ? ORACLE_ERR_NONFINITE : ORACLE_OK;
}

}  // namespace

extern "C" {

// Advances f (layout [nc][Q][nz][ny][nx], x fastest) by nsteps in place. Returns a status;
// on error f holds the state before the failing step and *failed_step its index (0-based).
int oracle_step(const oracle_case* c, double* f, int nsteps, int* failed_step) {
  Setup S;
  int st = make_setup(c, &S);
  if (st != ORACLE_OK) return st;
  std::vector<double> buf((size_t)S.nc * S.L.Q * S.N);
  double kij[16], gamma[4];
  for (int k = 0; k < 16; ++k) kij[k] = c->kij[k];
  for (int k = 0; k < 4; ++k) gamma[k] = c->gamma[k];
  for (int n = 0; n < nsteps; ++n) {
    st = step_once<double>(S, kij, gamma, f, buf.data());
    if (st != ORACLE_OK) {
      if (failed_step) *failed_step = n;
      return st;
    }
    std::memcpy(f, buf.data(), buf.size() * sizeof(double));
  }
  return ORACLE_OK;
}

// Same as oracle_step on dual numbers: f is [3][nc][Q][N] (value, d/dtheta0, d/dtheta1);
// dkij is [2][nc*nc] and dgamma [2][nc], the derivatives of zeta_ij and gamma_i with
// respect to the two parameters theta0, theta1.
int oracle_step_dual(const oracle_case* c, const double* dkij, const double* dgamma, double* f,
                     int nsteps, int* failed_step) {
  Setup S;
  int st = make_setup(c, &S);
  if (st != ORACLE_OK) return st;
  if (S.split != 0) return ORACLE_ERR_ARG;  // the dual path differentiates Eq. distributionforce
  const int nc = S.nc;
  const size_t n = (size_t)nc * S.L.Q * S.N;
  Dual kij[16], gamma[4];
  for (int k = 0; k < nc * nc; ++k) kij[k] = Dual(c->kij[k], dkij[k], dkij[nc * nc + k]);
  for (int k = 0; k < nc; ++k) gamma[k] = Dual(c->gamma[k], dgamma[k], dgamma[nc + k]);
  std::vector<Dual> a(n), b(n);
  for (size_t k = 0; k < n; ++k) a[k] = Dual(f[k], f[n + k], f[2 * n + k]);
  for (int s = 0; s < nsteps; ++s) {
    st = step_once<Dual>(S, kij, gamma, a.data(), b.data());
    if (st != ORACLE_OK) {
      if (failed_step) *failed_step = s;
      break;
    }
    a.swap(b);
  }
  for (size_t k = 0; k < n; ++k) {
    f[k] = a[k].v;
    f[n + k] = a[k].d0;
    f[2 * n + k] = a[k].d1;
  }
  return st;
}

// Macroscopic fields of state f: rho [nc][N], u [3][N] (barycentric, Guo half force),
// p [N] (EOS pressure), psi [N], F [3][N] (total force). Any output may be NULL.
int oracle_fields(const oracle_case* c, const double* f, double* rho, double* u, double* p,
                  double* psi, double* F) {
  Setup S;
  int st = make_setup(c, &S);
  if (st != ORACLE_OK) return st;
  double kij[16];
  for (int k = 0; k < 16; ++k) kij[k] = c->kij[k];
  Macro<double> m;
  st = macroscopic<double>(S, kij, f, m);
  if (st != ORACLE_OK) return st;
  const int64_t N = S.N;
  for (int64_t x = 0; x < N; ++x) {
    double r = 0;
    for (int s = 0; s < S.nc; ++s) {
      r += m.rho_c[s * N + x];
      if (rho) rho[s * N + x] = m.rho_c[s * N + x];
    }
    for (int d = 0; d < 3; ++d) {
      if (u) u[d * N + x] = (m.mom[d * N + x] + 0.5 * m.F[d * N + x]) / r;
      if (F) F[d * N + x] = m.F[d * N + x];
    }
    if (p) p[x] = m.p[x];
    if (psi) psi[x] = m.psi[x];
  }
  return ORACLE_OK;
}

// EOS pressure and psi^2 of one site from its cell-volume densities (for pins).
int oracle_eos(const oracle_case* c, const double* rho_c, double* p, double* psi2) {
  Setup S;
  int st = make_setup(c, &S);
  if (st != ORACLE_OK) return st;
  double kij[16];
  for (int k = 0; k < 16; ++k) kij[k] = c->kij[k];
  return eos<double>(S, kij, rho_c, p, psi2);
}

// Equilibrium populations f_eq(rho_s, u) of Eq. equilibrium(a): the initial state.
int oracle_equilibrium(const oracle_case* c, const double* rho, const double* u, double* f) {
  Setup S;
  int st = make_setup(c, &S);
  if (st != ORACLE_OK) return st;
  const int Q = S.L.Q, D = S.L.D;
  const int64_t N = S.N;
  for (int64_t x = 0; x < N; ++x) {
    double uu = 0, uv[3] = {0, 0, 0};
    for (int d = 0; d < D; ++d) {
      uv[d] = u ? u[d * N + x] : 0.0;
      uu += uv[d] * uv[d];
    }
    for (int s = 0; s < S.nc; ++s)
      for (int a = 0; a < Q; ++a) {
        double eu = 0;
        for (int d = 0; d < D; ++d) eu += S.L.e[a][d] * uv[d];
        f[((int64_t)s * Q + a) * N + x] =
            rho[s * N + x] * S.L.w[a] *
            (1 + eu / CS2 + eu * eu / (2 * CS2 * CS2) - uu / (2 * CS2));
      }
  }
  return ORACLE_OK;
}

// Threads the oracle's loops use (OpenMP; results do not depend on it).
int oracle_threads(void) { return omp_get_max_threads(); }

// Sets the threads of the oracle's later loops (the timed baseline runs it on one core and on
// all of them); n < 1 is ignored.
void oracle_set_threads(int n) {
  if (n >= 1) omp_set_num_threads(n);
}

// Lattice tables, exported for the tests' invariants (velocity e [19][3], weights [19]).
int oracle_lattice(int Q, int* e, double* w) {
  if (Q != 9 && Q != 19) return ORACLE_ERR_ARG;
  Lattice L = make_lattice(Q);
  for (int a = 0; a < Q; ++a) {
    for (int d = 0; d < 3; ++d) e[a * 3 + d] = L.e[a][d];
    w[a] = L.w[a];
  }
  return L.D;
}

// MRT matrix M [Q][Q] and its inverse, for the tests.
int oracle_mrt_matrix(int Q, double* M, double* Minv) {
  if (Q != 9 && Q != 19) return ORACLE_ERR_ARG;
  Lattice L = make_lattice(Q);
  for (int k = 0; k < Q; ++k)
    for (int a = 0; a < Q; ++a) M[k * Q + a] = moment_row(Q, k, L.e[a]);
  return invert(Q, M, Minv) ? ORACLE_OK : ORACLE_ERR_ARG;
}

}  // extern "C"
