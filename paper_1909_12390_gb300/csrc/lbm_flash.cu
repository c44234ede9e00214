// Batched two-phase flash of the Peng-Robinson mixture (Section 3.2): many (T, p, z) cases of
// one set of components, one FP64 thread per case. It produces the phase compositions, the
// compressibility factors, the phase densities and the volatility coefficients gamma_i that
// set up the multi-component runs (Section 4.2).
//
// Per case, following Section 3.2:
//   * A_i = Omega_a alpha_i p_ri / T_ri^2, B_i = Omega_b p_ri / T_ri (Eq. cubiccoeff; the
//     printed A_i has T_ri where T_ri^2 belongs), A_ij = sqrt(A_i A_j) (1 - zeta_ij),
//     A = sum c_i c_j A_ij, B = sum c_i B_i;
//   * the roots Z > B of Z^3 - (1 - B) Z^2 + (A - 3B^2 - 2B) Z - (AB - B^2 - B^3) = 0 (the cubic
//     that follows from Eq. MCPengRobinson; the printed Eq. PRcubic has two wrong
//     coefficients), by the trigonometric / Cardano closed form and Newton polishing;
//   * the root of lower Gibbs energy (Eq. solutionselection; dG = 0 takes the largest);
//   * ln phi_i of Eq. fugacitycoeff2;
//   * Wilson K_i to start, then successive substitution K_i = phi_li / phi_vi with the vapour
//     fraction from the Rachford-Rice equation (negative flash allowed), until
//     max_i |ln K_i^new - ln K_i| < tol;
//   * the iso-fugacity residual of Eq. error, n = p / (Z R T), rho_i = n x_i M_i per phase,
//     and gamma_i = ln(rho_il / rho_iv) / ln(rho_hl / rho_hv) with h the least volatile
//     component (smallest K), the per-component form of Eq. gamma.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <string>

#include "lbm.h"

namespace {

constexpr double kOmegaA = 0.45724;
constexpr double kOmegaB = 0.0778;
constexpr double kSqrt2 = 1.4142135623730950488;
constexpr int kMaxNc = 4;

struct FlashComp {
  double Tc[kMaxNc], pc[kMaxNc], omega[kMaxNc], M[kMaxNc];
};

__device__ double m_of(double w) {
  return w <= 0.49 ? 0.374640 + w * (1.54226 - 0.26992 * w)
                   : 0.379642 + w * (1.48503 + w * (-0.164423 + 0.016666 * w));
}

// Real roots Z > B of the PR cubic, ascending; returns their number (0..3).
__device__ int pr_roots(double A, double B, double* z) {
  const double a2 = -(1.0 - B), a1 = A - 3.0 * B * B - 2.0 * B, a0 = -(A * B - B * B - B * B * B);
  const double sh = a2 / 3.0;
  const double p = a1 - a2 * sh;                              // depressed cubic t^3 + p t + q
  const double q = 2.0 * sh * sh * sh - sh * a1 + a0;
  const double disc = 0.25 * q * q + p * p * p / 27.0;
  double r[3];
  int n;
  if (disc > 0.0) {
    const double s = sqrt(disc);
    r[0] = cbrt(-0.5 * q + s) + cbrt(-0.5 * q - s) - sh;
    n = 1;
  } else {
    const double rr = sqrt(fmax(-p / 3.0, 0.0));
    double c = rr > 0.0 ? -0.5 * q / (rr * rr * rr) : 0.0;
    c = fmin(1.0, fmax(-1.0, c));
    const double ph = acos(c) / 3.0;
    const double tp = 2.0943951023931954923;  // 2 pi / 3
    r[0] = 2.0 * rr * cos(ph) - sh;
    r[1] = 2.0 * rr * cos(ph - tp) - sh;
    r[2] = 2.0 * rr * cos(ph + tp) - sh;
    n = 3;
  }
  int m = 0;
  for (int k = 0; k < n; ++k) {
    double x = r[k];
    for (int it = 0; it < 3; ++it) {  // Newton polishing on the original cubic
      const double f = ((x + a2) * x + a1) * x + a0;
      const double d = (3.0 * x + 2.0 * a2) * x + a1;
      if (d != 0.0) x -= f / d;
    }
    if (x > B) z[m++] = x;
  }
  for (int i = 1; i < m; ++i)  // ascending
    for (int j = i; j > 0 && z[j] < z[j - 1]; --j) {
      const double t = z[j];
      z[j] = z[j - 1];
      z[j - 1] = t;
    }
  return m;
}

struct Coef {
  double Ai[kMaxNc], Bi[kMaxNc];
};

// Z and ln phi_i of one phase of composition c (root chosen by Gibbs energy); false if the
// cubic has no root above B.
__device__ bool phase(int nc, const Coef& k, const double* kij, const double* c, double& Z, double* lnphi) {
  double s[kMaxNc], A = 0.0, B = 0.0;
  for (int i = 0; i < nc; ++i) {
    s[i] = 0.0;
    for (int j = 0; j < nc; ++j) s[i] += sqrt(k.Ai[i] * k.Ai[j]) * (1.0 - kij[i * nc + j]) * c[j];
    A += c[i] * s[i];
    B += c[i] * k.Bi[i];
  }
  double z[3];
  const int m = pr_roots(A, B, z);
  if (m == 0) return false;
  Z = z[0];
  if (m > 1) {
    const double zl = z[0], zv = z[m - 1];
    const double dG = (zv - zl) + log((zl - B) / (zv - B)) +
                      A / (2.0 * kSqrt2 * B) *
                          log(((zl + (1.0 + kSqrt2) * B) * (zv + (1.0 - kSqrt2) * B)) /
                              ((zl + (1.0 - kSqrt2) * B) * (zv + (1.0 + kSqrt2) * B)));
    Z = dG > 0.0 ? zl : zv;
  }
  const double lg = log((Z + (1.0 - kSqrt2) * B) / (Z + (1.0 + kSqrt2) * B));
  for (int i = 0; i < nc; ++i)
    lnphi[i] = -log(Z - B) + k.Bi[i] / B * (Z - 1.0) + A / (2.0 * kSqrt2 * B) * (2.0 * s[i] / A - k.Bi[i] / B) * lg;
  return true;
}

// Vapour fraction solving sum z_i (K_i - 1) / (1 + V (K_i - 1)) = 0 between the poles, by
// Newton steps kept inside a shrinking bracket; false if all K_i lie on one side of 1.
__device__ bool rachford_rice(int nc, const double* z, const double* K, double& V) {
  double kmax = K[0], kmin = K[0];
  for (int i = 1; i < nc; ++i) {
    kmax = fmax(kmax, K[i]);
    kmin = fmin(kmin, K[i]);
  }
  if (kmax <= 1.0 || kmin >= 1.0) return false;
  double lo = 1.0 / (1.0 - kmax), hi = 1.0 / (1.0 - kmin);  // g > 0 near lo, < 0 near hi
  double v = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double g = 0.0, dg = 0.0;
    for (int i = 0; i < nc; ++i) {
      const double km = K[i] - 1.0, den = 1.0 + v * km;
      g += z[i] * km / den;
      dg -= z[i] * km * km / (den * den);
    }
    if (g > 0.0)
      lo = v;
    else
      hi = v;
    double nv = dg != 0.0 ? v - g / dg : 0.5 * (lo + hi);
    if (!(nv > lo && nv < hi)) nv = 0.5 * (lo + hi);
    if (nv == v || hi - lo <= 4e-16 * fmax(1.0, fabs(v))) {
      v = nv;
      break;
    }
    v = nv;
  }
  V = v;
  return true;
}

__global__ void k_flash(int nc, FlashComp cp, int ncase, const lbm_flash_case* __restrict__ cases,
                        lbm_flash_result* __restrict__ out, double R, double tol, int maxit) {
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  if (ci >= ncase) return;
  const lbm_flash_case cs = cases[ci];
  lbm_flash_result r{};
  const double T = cs.T, p = cs.p;
  Coef k;
  double K[kMaxNc], z[kMaxNc], x[kMaxNc], y[kMaxNc];
  for (int i = 0; i < nc; ++i) {
    const double Tr = T / cp.Tc[i], pr = p / cp.pc[i];
    const double al = 1.0 + m_of(cp.omega[i]) * (1.0 - sqrt(Tr));
    k.Ai[i] = kOmegaA * al * al * pr / (Tr * Tr);
    k.Bi[i] = kOmegaB * pr / Tr;
    K[i] = cp.pc[i] / p * exp(5.373 * (1.0 + cp.omega[i]) * (1.0 - cp.Tc[i] / T));  // Wilson
    z[i] = cs.z[i];
    x[i] = y[i] = z[i];
  }
  double V = 0.0, Zl = 0.0, Zv = 0.0, lpl[kMaxNc], lpv[kMaxNc];
  bool two = false, conv = false;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    if (!rachford_rice(nc, z, K, V)) break;
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < nc; ++i) {
      x[i] = z[i] / (1.0 + V * (K[i] - 1.0));
      y[i] = K[i] * x[i];
      sx += x[i];
      sy += y[i];
    }
    for (int i = 0; i < nc; ++i) {
      x[i] /= sx;
      y[i] /= sy;
    }
    if (!phase(nc, k, cs.kij, x, Zl, lpl) || !phase(nc, k, cs.kij, y, Zv, lpv)) break;
    two = true;
    double step = 0.0;
    for (int i = 0; i < nc; ++i) {
      const double lk = lpl[i] - lpv[i];
      step = fmax(step, fabs(lk - log(K[i])));
      K[i] = exp(lk);
    }
    if (step < tol) {
      conv = true;
      break;
    }
  }
  double kdev = 0.0;
  for (int i = 0; i < nc; ++i) kdev = fmax(kdev, fabs(log(K[i])));
  const bool trivial = !two || kdev < 1e-4;
  r.V = V;
  r.Zl = Zl;
  r.Zv = Zv;
  r.iterations = it > maxit ? maxit : it;
  r.status = trivial ? 1 : (conv ? 0 : 2);
  for (int i = 0; i < nc; ++i) {
    r.x[i] = x[i];
    r.y[i] = y[i];
    r.K[i] = K[i];
  }
  r.residual = NAN;
  if (!trivial) {
    // iso-fugacity residual at the final compositions, f_i = phi_i c_i p
    double zl, zv;
    if (phase(nc, k, cs.kij, x, zl, lpl) && phase(nc, k, cs.kij, y, zv, lpv)) {
      double res = 0.0;
      for (int i = 0; i < nc; ++i) {
        const double q = exp(lpl[i] - lpv[i]) * x[i] / y[i] - 1.0;
        res += q * q;
      }
      r.residual = res;
    }
    const double nl = p / (Zl * R * T), nv = p / (Zv * R * T);
    int h = 0;
    for (int i = 1; i < nc; ++i)
      if (K[i] < K[h]) h = i;
    for (int i = 0; i < nc; ++i) {
      r.rho_l[i] = nl * x[i] * cp.M[i];
      r.rho_v[i] = nv * y[i] * cp.M[i];
    }
    const double den = log(r.rho_l[h] / r.rho_v[h]);
    for (int i = 0; i < nc; ++i) r.gamma[i] = log(r.rho_l[i] / r.rho_v[i]) / den;
  }
  out[ci] = r;
}

thread_local char g_flash_msg[256];

lbm_status flash_fail(lbm_status st, const char* what) {
  snprintf(g_flash_msg, sizeof g_flash_msg, "%s", what);
  return st;
}

}  // namespace

extern "C" {

lbm_status lbm_flash(int nc, const lbm_component* comps, int ncase, const lbm_flash_case* cases, double R,
                     double tol, int maxit, void* stream, lbm_flash_result* out) {
  g_flash_msg[0] = 0;
  if (nc < 1 || nc > kMaxNc) return flash_fail(LBM_ERR_ARG, "nc must be 1..4");
  if (!comps || !cases || !out) return flash_fail(LBM_ERR_ARG, "comps, cases and out must be non-NULL");
  if (ncase < 0) return flash_fail(LBM_ERR_ARG, "ncase must be >= 0");
  if (!(tol > 0) || maxit < 1) return flash_fail(LBM_ERR_ARG, "tol must be > 0 and maxit >= 1");
  if (!(R > 0) || !std::isfinite(R)) return flash_fail(LBM_ERR_ARG, "R must be finite and > 0");
  FlashComp cp{};
  for (int i = 0; i < nc; ++i) {
    const lbm_component& c = comps[i];
    if (!(c.Tc > 0) || !(c.pc > 0) || !(c.M > 0) || !std::isfinite(c.omega))
      return flash_fail(LBM_ERR_ARG, "components need Tc, pc, M > 0 and a finite omega");
    cp.Tc[i] = c.Tc;
    cp.pc[i] = c.pc;
    cp.omega[i] = c.omega;
    cp.M[i] = c.M;
  }
  for (int j = 0; j < ncase; ++j) {
    const lbm_flash_case& cs = cases[j];
    double s = 0.0;
    bool ok = cs.T > 0 && cs.p > 0 && std::isfinite(cs.T) && std::isfinite(cs.p);
    for (int i = 0; i < nc; ++i) {
      ok = ok && cs.z[i] > 0 && std::isfinite(cs.z[i]);
      s += cs.z[i];
      for (int l = 0; l < nc; ++l) ok = ok && std::isfinite(cs.kij[i * nc + l]) && cs.kij[i * nc + l] == cs.kij[l * nc + i];
    }
    if (!ok || std::fabs(s - 1.0) > 1e-9) {
      char m[160];
      snprintf(m, sizeof m, "case %d: T, p > 0, z_i > 0 summing to 1 and a symmetric finite kij are required", j);
      return flash_fail(LBM_ERR_ARG, m);
    }
  }
  if (ncase == 0) return LBM_OK;
  cudaStream_t s = (cudaStream_t)stream;
  lbm_flash_case* d_cases = nullptr;
  lbm_flash_result* d_out = nullptr;
  cudaError_t e = cudaMallocAsync(&d_cases, sizeof(lbm_flash_case) * ncase, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_out, sizeof(lbm_flash_result) * ncase, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cases, cases, sizeof(lbm_flash_case) * ncase, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_flash<<<(ncase + 127) / 128, 128, 0, s>>>(nc, cp, ncase, d_cases, d_out, R, tol, maxit);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(lbm_flash_result) * ncase, cudaMemcpyDeviceToHost, s);
  if (d_cases) cudaFreeAsync(d_cases, s);
  if (d_out) cudaFreeAsync(d_out, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    char m[200];
    snprintf(m, sizeof m, "CUDA: %s", cudaGetErrorString(e));
    return flash_fail(LBM_ERR_CUDA, m);
  }
  return LBM_OK;
}

const char* lbm_flash_error(void) { return g_flash_msg; }

}  // extern "C"
